// Per-view preprocessing, count scan and pair emission (sm_103a).
//
//   k_tile_mask   per 8x4 pixel block and per tile: OR of 1 << signbits(r_d)
//                 over the in-image pixels
//                 (ray sign bits of Sec. B.2; duplication per sign pattern,
//                 Sec. B.1)
//   k_preprocess  per (view, voxel): lattice index, Morton code (Sec. A.1),
//                 tile rectangle of the projected corners (Sec. 3.1.2), pair
//                 count, conservative pixel box, view-dependent colour
//                 (Eq. vox_color), gathered densities
//                 and, per tile, the pairs it will hold (atomics);
//                 k_preprocess_views does the same for a batch of views with
//                 one thread per voxel, reading its densities and SH once
//   k_scan_*      exclusive scan of the tiles' pair counts (block sums, then
//                 each block scans its part after summing the earlier blocks;
//                 kTileSub sub-buckets per tile, adjacent): each sub-bucket's
//                 start, each tile's end, the total, the capacity check
//   k_emit        writes each (voxel, tile, sign pattern s) pair into its
//                 tile's range (an atomic cursor per sub-bucket; the order
//                 within a tile is left to the per-tile sort):
//                 key = tile << S | top S bits of (octpath ^ s replicated),
//                 value = s << 29 | voxel id (Sec. B.1; the per-triple
//                 permutation of Sec. B.2 is b ^ s, applied to all 16
//                 triples at once).  S = 48 for one view (the paper's layout:
//                 16-bit tile id over the 48-bit order); a batch of views uses
//                 the global tile id over the 3 (max_level + 1) Morton bits
//                 that can differ, so more than 2^16 tiles fit in 64 bits.
#include <climits>

#include "svr_internal.cuh"

namespace svr {

// --------------------------------------------------------------- tile masks

// One warp per tile, looping over its 8x4 pixel blocks (the render's warp
// blocks, tile / 8 per block row): each block's sign-bit mask goes to
// block_sign, their OR to tile_mask.
constexpr int kMaskWarps = 8;

__global__ void __launch_bounds__(32 * kMaskWarps) k_tile_mask(FrameDev f) {
    // also starts the frame: status cleared (no smallest invalid voxel yet)
    // and the tiles' pair counters zeroed, before k_preprocess counts
    if (blockIdx.x == 0 && threadIdx.x < sizeof(Status) / 4)
        reinterpret_cast<unsigned *>(f.status)[threadIdx.x] =
            threadIdx.x == offsetof(Status, bad_voxel) / 4 ? 0xFFFFFFFFu : 0u;
    const int g = blockIdx.x * kMaskWarps + (threadIdx.x >> 5);
    if (g >= f.total_tiles) return;
    if ((threadIdx.x & 31) < kTileSub) f.tile_cnt[(size_t)(threadIdx.x & 31) * f.total_tiles + g] = 0u;
    const DevCam &cam = f.views[view_of_tile(f, g)];
    const int tile = g - cam.tile_base;
    const int T = cam.tile, bpr = T >> 3, B = f.blocks_per_tile;
    const int x0 = (tile % cam.ntx) * T, y0 = (tile / cam.ntx) * T;
    const int lane = threadIdx.x & 31;
    unsigned m = 0;
    for (int b = 0; b < B; ++b) {
        const int x = x0 + (b % bpr) * 8 + (lane & 7), y = y0 + (b / bpr) * 4 + (lane >> 3);
        const unsigned bit = (x < cam.W && y < cam.H) ? 1u << sign_bits(pixel_dir(cam, x, y)) : 0u;
        const unsigned bm = __reduce_or_sync(0xffffffffu, bit);
        if (lane == b) f.block_sign[(size_t)g * B + b] = (uint8_t)bm;
        m |= bm;
    }
    if (lane == 0) f.tile_mask[g] = (uint8_t)m;
}

// --------------------------------------------------------------- preprocess

// Spread the low 16 bits of x to bit positions 0, 3, 6, ..., 45.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0xFFFFu;
    x = (x | (x << 16)) & 0x0000FF0000FFull;
    x = (x | (x << 8)) & 0x00F00F00F00Full;
    x = (x | (x << 4)) & 0x0C30C30C30C3ull;
    x = (x | (x << 2)) & 0x249249249249ull;
    return x;
}

__device__ __forceinline__ void mark_invalid(Status *st, int64_t v) {
    atomicOr(&st->flags, SVR_FLAG_INVALID_VOXEL);
    atomicMin(reinterpret_cast<unsigned *>(&st->bad_voxel), (unsigned)v);
}

// Lattice index of voxel v (centre = w_min + v_s (ijk + 1/2)) and the
// validity of its level, centre and corner indices.
__device__ __forceinline__ bool voxel_valid(const FrameDev &f, int64_t v, float c0, float c1, float c2, int l,
                                            float &vs, int ijk[3], int4 &i0, int4 &i1) {
    bool ok = l >= 1 && l <= f.max_level;
    vs = ldexpf(f.world_size, -l);
    ijk[0] = ijk[1] = ijk[2] = 0;
    if (ok) {
        const float cc[3] = {c0, c1, c2};
        const int n = 1 << l;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float fi = (cc[a] - f.world_min[a]) / vs - 0.5f;
            float r = rintf(fi);
            ok = ok && fabsf(fi - r) <= 0.25f && r >= 0.f && r < (float)n;
            ijk[a] = (int)r;
        }
    }
    // corner indices must name grid points
    const int4 *ci = reinterpret_cast<const int4 *>(f.corner_idx + 8 * v);
    i0 = __ldg(ci);
    i1 = __ldg(ci + 1);
    const int64_t np = f.n_pts;
    const int lo = min(min(min(i0.x, i0.y), min(i0.z, i0.w)), min(min(i1.x, i1.y), min(i1.z, i1.w)));
    const int hi = max(max(max(i0.x, i0.y), max(i0.z, i0.w)), max(max(i1.x, i1.y), max(i1.z, i1.w)));
    return ok && lo >= 0 && (int64_t)hi < np;
}

// Projection of voxel v in one view: tile rectangle, conservative pixel box
// and pair count (the tiles' counts raised by atomics); writes rect and
// count of (view, voxel) iv and returns the count.
__device__ __forceinline__ uint32_t project_voxel(const FrameDev &f, const DevCam &cam, int64_t v, int64_t iv,
                                                  float c0, float c1, float c2, float h, ushort4 &box) {
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    int behind = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float px = (c & 4) ? c0 + h : c0 - h;
        const float py = (c & 2) ? c1 + h : c1 - h;
        const float pz = (c & 1) ? c2 + h : c2 - h;
        const float X = fmaf(cam.R[0], px, fmaf(cam.R[1], py, fmaf(cam.R[2], pz, cam.t[0])));
        const float Y = fmaf(cam.R[3], px, fmaf(cam.R[4], py, fmaf(cam.R[5], pz, cam.t[1])));
        const float Z = fmaf(cam.R[6], px, fmaf(cam.R[7], py, fmaf(cam.R[8], pz, cam.t[2])));
        if (Z <= kNear) {
            ++behind;
        } else {
            const float u = fmaf(cam.fx, X / Z, cam.cx);
            const float w = fmaf(cam.fy, Y / Z, cam.cy);
            umin = fminf(umin, u);
            umax = fmaxf(umax, u);
            vmin = fminf(vmin, w);
            vmax = fmaxf(vmax, w);
        }
    }
    short4 rc = make_short4(0, -1, 0, -1);
    box = make_ushort4(0, (unsigned short)(cam.W - 1), 0, (unsigned short)(cam.H - 1));
    if (behind == 8) {
        // culled
    } else if (behind > 0) {
        rc = make_short4(0, (short)(cam.ntx - 1), 0, (short)(cam.nty - 1));
    } else if (!(umax < 0.f || umin >= (float)cam.W || vmax < 0.f || vmin >= (float)cam.H)) {
        // pixels whose centre (x + 1/2, y + 1/2) can lie in the projected box,
        // widened by a rounding margin: a conservative filter for the render
        const float mu = 0.01f + 1e-5f * fmaxf(fabsf(umin), fabsf(umax));
        const float mv = 0.01f + 1e-5f * fmaxf(fabsf(vmin), fabsf(vmax));
        const float fx0 = fmaxf(floorf(umin - 0.5f - mu), 0.f), fx1 = fminf(floorf(umax - 0.5f + mu), (float)(cam.W - 1));
        const float fy0 = fmaxf(floorf(vmin - 0.5f - mv), 0.f), fy1 = fminf(floorf(vmax - 0.5f + mv), (float)(cam.H - 1));
        box = make_ushort4((unsigned short)fx0, (unsigned short)fmaxf(fx1, fx0), (unsigned short)fy0,
                           (unsigned short)fmaxf(fy1, fy0));
        const float T = (float)cam.tile;
        const int tx0 = umin < 0.f ? 0 : min(cam.ntx - 1, (int)floorf(umin / T));
        const int tx1 = umax >= (float)cam.W ? cam.ntx - 1 : min(cam.ntx - 1, (int)floorf(umax / T));
        const int ty0 = vmin < 0.f ? 0 : min(cam.nty - 1, (int)floorf(vmin / T));
        const int ty1 = vmax >= (float)cam.H ? cam.nty - 1 : min(cam.nty - 1, (int)floorf(vmax / T));
        rc = make_short4((short)tx0, (short)tx1, (short)ty0, (short)ty1);
    }
    uint32_t cnt = 0;
    const uint8_t *mask = f.tile_mask + cam.tile_base;
    for (int ty = rc.z; ty <= rc.w; ++ty) {
        for (int tx = rc.x; tx <= rc.y; ++tx) {
            const uint32_t c = __popc(mask[ty * cam.ntx + tx]);
            if (c)
                atomicAdd(f.tile_cnt + (size_t)(v & (kTileSub - 1)) * f.total_tiles + cam.tile_base + ty * cam.ntx + tx,
                          c);
            cnt += c;
        }
    }
    f.rect[iv] = rc;
    f.count[iv] = cnt;
    return cnt;
}

// Colour of the voxel in one view (Eq. vox_color): degree-3 SH at the
// direction from the view's ray origin to the centre, clamped at 0; bit c of
// the w word set if channel c was > 0 before the clamp.
__device__ __forceinline__ void view_basis(const DevCam &cam, float c0, float c1, float c2, float Y[16]) {
    float dx = c0 - cam.ro[0], dy = c1 - cam.ro[1], dz = c2 - cam.ro[2];
    const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv;
    dy *= inv;
    dz *= inv;
    sh_basis(dx, dy, dz, Y);
}

__device__ __forceinline__ float4 voxel_colour(const float Y[16], const float sh[48]) {
    float col[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.f;
#pragma unroll
        for (int n = 0; n < 16; ++n) acc = fmaf(Y[n], sh[3 * n + ch], acc);
        col[ch] = acc;
    }
    const unsigned bits = (col[0] > 0.f ? 1u : 0u) | (col[1] > 0.f ? 2u : 0u) | (col[2] > 0.f ? 4u : 0u);
    return make_float4(fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f), __uint_as_float(bits));
}

__device__ __forceinline__ void load_sh(const FrameDev &f, int64_t v, float sh[48]) {
    const float4 *shv = reinterpret_cast<const float4 *>(f.sh + 48 * v);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const float4 s4 = __ldg(shv + q);
        sh[4 * q + 0] = s4.x;
        sh[4 * q + 1] = s4.y;
        sh[4 * q + 2] = s4.z;
        sh[4 * q + 3] = s4.w;
    }
}

__device__ __forceinline__ void write_octpath(const FrameDev &f, int64_t v, int l, const int ijk[3]) {
    f.octpath[v] = ((spread3(ijk[0]) << 2) | (spread3(ijk[1]) << 1) | spread3(ijk[2])) << (3 * (kMaxLevel - l));
}

// One view (grid.y = view): one thread per (view, voxel).
__global__ void __launch_bounds__(128, 8) k_preprocess(FrameDev f) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= f.n_vox) return;
    const int view = blockIdx.y;
    const DevCam &cam = f.views[view];
    const int64_t iv = (int64_t)view * f.n_vox + v;
    const float c0 = f.centre[3 * v + 0], c1 = f.centre[3 * v + 1], c2 = f.centre[3 * v + 2];
    const int l = f.level[v];
    float vs;
    int ijk[3];
    int4 i0, i1;
    if (!voxel_valid(f, v, c0, c1, c2, l, vs, ijk, i0, i1)) {
        if (view == 0) mark_invalid(f.status, v);
        f.count[iv] = 0;
        f.rect[iv] = make_short4(0, -1, 0, -1);
        return;
    }
    if (view == 0) write_octpath(f, v, l, ijk);
    const float h = 0.5f * vs;
    ushort4 box;
    if (project_voxel(f, cam, v, iv, c0, c1, c2, h, box) == 0) return;
    f.box[iv] = box;
    // record of this view: min corner relative to the ray origin, size,
    // gathered raw densities, colour
    Record r;
    r.r0 = make_float4((c0 - h) - cam.ro[0], (c1 - h) - cam.ro[1], (c2 - h) - cam.ro[2], vs);
    r.r1 = make_float4(__ldg(f.grid + i0.x), __ldg(f.grid + i0.y), __ldg(f.grid + i0.z), __ldg(f.grid + i0.w));
    r.r2 = make_float4(__ldg(f.grid + i1.x), __ldg(f.grid + i1.y), __ldg(f.grid + i1.z), __ldg(f.grid + i1.w));
    float Y[16], sh[48];
    view_basis(cam, c0, c1, c2, Y);
    load_sh(f, v, sh);
    r.r3 = voxel_colour(Y, sh);
    f.rec[iv] = r;
}

// Several views: one thread per voxel.  The voxel's validity, Morton code,
// densities and SH coefficients are read once for all views (the SH only
// while the views' colours are evaluated, which are written first, into the
// records' colour words); then each view's projection, tile counts and the
// rest of its record.
__global__ void __launch_bounds__(128) k_preprocess_views(FrameDev f) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= f.n_vox) return;
    const float c0 = f.centre[3 * v + 0], c1 = f.centre[3 * v + 1], c2 = f.centre[3 * v + 2];
    const int l = f.level[v];
    float vs;
    int ijk[3];
    int4 i0, i1;
    if (!voxel_valid(f, v, c0, c1, c2, l, vs, ijk, i0, i1)) {
        mark_invalid(f.status, v);
        for (int view = 0; view < f.n_views; ++view) {
            const int64_t iv = (int64_t)view * f.n_vox + v;
            f.count[iv] = 0;
            f.rect[iv] = make_short4(0, -1, 0, -1);
        }
        return;
    }
    write_octpath(f, v, l, ijk);
    {
        float sh[48];
        load_sh(f, v, sh);
        for (int view = 0; view < f.n_views; ++view) {
            float Y[16];
            view_basis(f.views[view], c0, c1, c2, Y);
            f.rec[(int64_t)view * f.n_vox + v].r3 = voxel_colour(Y, sh);
        }
    }
    const float4 g0 = make_float4(__ldg(f.grid + i0.x), __ldg(f.grid + i0.y), __ldg(f.grid + i0.z), __ldg(f.grid + i0.w));
    const float4 g1 = make_float4(__ldg(f.grid + i1.x), __ldg(f.grid + i1.y), __ldg(f.grid + i1.z), __ldg(f.grid + i1.w));
    const float h = 0.5f * vs;
    for (int view = 0; view < f.n_views; ++view) {
        const DevCam &cam = f.views[view];
        const int64_t iv = (int64_t)view * f.n_vox + v;
        ushort4 box;
        if (project_voxel(f, cam, v, iv, c0, c1, c2, h, box) == 0) continue;
        f.box[iv] = box;
        Record *r = f.rec + iv;
        r->r0 = make_float4((c0 - h) - cam.ro[0], (c1 - h) - cam.ro[1], (c2 - h) - cam.ro[2], vs);
        r->r1 = g0;
        r->r2 = g1;
    }
}

// --------------------------------------------------------------------- scan

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *warp_sums, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint32_t s = warp_sums[w];
        wpre += (w < warp) ? s : 0u;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return wpre + inc - x;
}

// Scan position i is sub-bucket i % kTileSub of tile i / kTileSub, stored
// sub-bucket-major (count[sub * ntiles + tile]).
__device__ __forceinline__ int64_t sub_index(int64_t i, int64_t ntiles) {
    return (i % kTileSub) * ntiles + i / kTileSub;
}

__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t *__restrict__ count, int64_t ntiles,
                                                     uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t ws[8];
    const int64_t n = ntiles * kTileSub;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint64_t acc = 0;
    for (int r = 0; r < kScanTile / 256; ++r) {
        int64_t i = base + r * 256 + threadIdx.x;
        if (i < n) acc += count[sub_index(i, ntiles)];
    }
    uint32_t tot;
    // a block sum beyond 2^32 saturates; the capacity check on the 64-bit
    // total catches it
    block_exclusive_scan((uint32_t)tmin<uint64_t>(acc, 0xFFFFFFFFull), ws, tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Sub-bucket starts (the emission cursors) and tile ends from the counts;
// k_tile_order turns them into the tiles' ranges.  Each CTA first sums the
// block sums of all earlier CTAs (64-bit), so no separate top-level scan is
// launched; the last CTA records the total and checks it against the
// capacity.  A start beyond 2^32 saturates; the capacity flag covers it.
__global__ void __launch_bounds__(256) k_scan_down(const uint32_t *__restrict__ count, int64_t ntiles,
                                                   const uint32_t *__restrict__ block_sums, int nb,
                                                   uint32_t *__restrict__ cursor, uint32_t *__restrict__ tile_end,
                                                   Status *st, int64_t capacity) {
    __shared__ uint32_t ws[8];
    __shared__ unsigned long long wpre[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long pre = 0;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += 256) pre += block_sums[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
    if (lane == 0) wpre[warp] = pre;
    __syncthreads();
    pre = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) pre += wpre[w];
    const int64_t n = ntiles * kTileSub;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    unsigned long long carry = pre;
    for (int r = 0; r < kScanTile / 256; ++r) {
        const int64_t i = base + r * 256 + threadIdx.x;
        const uint32_t x = i < n ? count[sub_index(i, ntiles)] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(x, ws, tot);
        if (i < n) {
            const uint32_t c = (uint32_t)tmin<unsigned long long>(carry + ex, 0xFFFFFFFFull);
            cursor[sub_index(i, ntiles)] = c;
            if (i % kTileSub == kTileSub - 1)
                tile_end[i / kTileSub] = (uint32_t)tmin<unsigned long long>(carry + ex + x, 0xFFFFFFFFull);
        }
        carry += tot;
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) {
        st->n_pairs_lo = (unsigned)(carry & 0xFFFFFFFFull);
        st->n_pairs_hi = (unsigned)(carry >> 32);
        if (carry > (unsigned long long)capacity) atomicOr(&st->flags, SVR_FLAG_CAPACITY);
    }
}

// --------------------------------------------------------------------- emit

constexpr int kEmitBatch = 8;
constexpr int kEmitThreads = 256;

// grid.y = view
__global__ void __launch_bounds__(kEmitThreads) k_emit(FrameDev f) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= f.n_vox) return;
    if (f.status->flags & SVR_FLAG_CAPACITY) return;
    const int view = blockIdx.y;
    const DevCam &cam = f.views[view];
    const int64_t iv = (int64_t)view * f.n_vox + v;
    if (f.count[iv] == 0) return;
    const short4 rc = f.rect[iv];
    const uint64_t code = f.octpath[v];
    const int drop = 48 - f.key_shift;
    uint64_t *keys = f.keys[0];
    uint32_t *vals = f.vals[0];
    uint32_t *cur = f.cursor + (size_t)(v & (kTileSub - 1)) * f.total_tiles;
    // the rectangle's tiles in row-major batches of kEmitBatch: a batch's
    // cursor atomics are issued together, so a voxel over many tiles waits
    // for one atomic round trip per batch rather than per tile
    int tx = rc.x, ty = rc.z;
    while (ty <= rc.w) {
        int gb[kEmitBatch];
        unsigned mb[kEmitBatch];
#pragma unroll
        for (int i = 0; i < kEmitBatch; ++i) {
            gb[i] = cam.tile_base + ty * cam.ntx + tx;
            mb[i] = ty <= rc.w && SVR_IN_BOUNDS(f.debug, kDbgTile, gb[i], f.total_tiles) ? (unsigned)f.tile_mask[gb[i]]
                                                                                   : 0u;
            if (++tx > rc.y) {
                tx = rc.x;
                ++ty;
            }
        }
        uint32_t ob[kEmitBatch];
#pragma unroll
        for (int i = 0; i < kEmitBatch; ++i) ob[i] = mb[i] ? atomicAdd(cur + gb[i], (uint32_t)__popc(mb[i])) : 0u;
#pragma unroll
        for (int i = 0; i < kEmitBatch; ++i) {
            unsigned m = mb[i];
            uint32_t o = ob[i];
            if ((int64_t)o + __popc(m) > f.capacity) {  // counts and emission disagree: never expected
                atomicOr(&f.status->flags, SVR_FLAG_CAPACITY);
                return;
            }
            while (m) {
                const unsigned s = __ffs(m) - 1;
                m &= m - 1;
                keys[o] = ((uint64_t)gb[i] << f.key_shift) | ((code ^ ((uint64_t)s * kTripleOnes)) >> drop);
                vals[o] = (s << 29) | (uint32_t)v;
                ++o;
            }
        }
    }
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_tile_mask(const FrameDev &f, cudaStream_t s) {
    k_tile_mask<<<(unsigned)((f.total_tiles + kMaskWarps - 1) / kMaskWarps), 32 * kMaskWarps, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_preprocess(const FrameDev &f, cudaStream_t s) {
    if (f.n_vox == 0) return cudaSuccess;
    if (f.n_views == 1) {
        k_preprocess<<<(unsigned)((f.n_vox + 127) / 128), 128, 0, s>>>(f);
    } else {
        k_preprocess_views<<<(unsigned)((f.n_vox + 127) / 128), 128, 0, s>>>(f);
    }
    return cudaGetLastError();
}

cudaError_t launch_scan(const FrameDev &f, cudaStream_t s) {
    const int64_t T = f.total_tiles;
    const int nb = (int)((T * kTileSub + kScanTile - 1) / kScanTile);
    k_scan_reduce<<<nb, 256, 0, s>>>(f.tile_cnt, T, f.scan_blocks);
    k_scan_down<<<nb, 256, 0, s>>>(f.tile_cnt, T, f.scan_blocks, nb, f.cursor, f.tile_end, f.status, f.capacity);
    return cudaGetLastError();
}

cudaError_t launch_emit(const FrameDev &f, cudaStream_t s) {
    if (f.n_vox > 0) {
        const dim3 grid((unsigned)((f.n_vox + kEmitThreads - 1) / kEmitThreads), (unsigned)f.n_views);
        k_emit<<<grid, kEmitThreads, 0, s>>>(f);
    }
    return cudaGetLastError();
}

}  // namespace svr
