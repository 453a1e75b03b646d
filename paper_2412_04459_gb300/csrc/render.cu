// Forward and backward compositing of the sorted tile lists (sm_103a).
//
// Work is split into items of (tile, list segment, 8x4 pixel block): 8
// blocks per 16x16 tile, and one segment per tile unless its list is longer
// than kSegLen entries.  A persistent grid of warps pulls items from a device
// counter in the order of k_tile_order (longest segments first, so the heavy
// work does not form the tail).  A warp walks the part of its block's list
// (the tile's entries whose pixel box meets the block, k_block_lists) that its
// segment covers, 32 entries per batch, with no CTA-wide barrier: lane j
// reads entry j of the batch (its value, then the voxel's conservative pixel
// box) and stages it into the warp's shared memory slots from the voxel's
// 64-byte record.
//
// Each batch then runs in two phases.  Phase A: lane j turns entry j into the
// mask of the block's pixels that may hit it (inside its pixel box and with
// its ray sign bits, Sec. B.1); a 32 x 32 bit transpose across the warp gives
// every pixel the mask of its candidate entries, and the pixel runs the
// ray-AABB slab test of Sec. A.2 on those only (entry and exit planes follow
// from the sign bits: 6 multiplies by 1/r_d and 4 min/max), recording its
// hits as a bit mask.  Phase B: in rounds, every pixel with hits left
// composites its next hit, so the lanes of a warp run the costly per-hit
// arithmetic together instead of one voxel at a time.
//
// The segments of a split list are walked from T = 1 by separate warps; the
// last of them to finish merges them front to back (exact up to rounding
// order, with a second walk of the segment in which a pixel stops) and leaves
// each segment's transmittance and the sums behind it for the backward.
//
// Forward (Sec. 3.1.2, Eq. alpha_blend, Eq. supp_alpha_comp, Sec. A.4):
//   K samples per segment, trilinear raw density, explin, per-sample
//   e_k = exp(-(l/K) explin(v_k)); 1 - alpha = prod_k e_k; local depth
//   d = sum_k prod_{j<k} e_j (1 - e_k) t_k; C += T alpha c, D += T d,
//   T *= 1 - alpha; a pixel stops after the voxel that leaves T < t_stop and
//   the warp leaves the list once all its pixels stopped.
//
// Backward, back to front from the saved (T_final, last).  With x_i the
// optical depth of voxel i (T_{i+1} = T_i exp(-x_i)) and, accumulated from
// the back, SC_i = sum_{j>i} T_j alpha_j c_j + T_final bg and
// SD_i = sum_{j>i} T_j d_j:
//   dC/dx_i = T_{i+1} c_i - SC_i,  dA/dx_i = T_final,  dD/dx_i|_T = -SD_i,
//   dC/dc_i = T_i alpha_i,
//   dd_i/dx_ik = P_{k+1} t_k - sum_{m>k} P_m (1 - e_m) t_m  (P_k = prod_{j<k} e_j;
//                the general form of the K <= 3 closed forms of Sec. A.4),
//   dx_ik/dv_k = (l/K) explin'(v_k), dv_k/dV_c = trilinear weight of corner c.
// T_i is recovered as T_{i+1} / exp(-x_i).  Pixels whose T_final is below
// 1e-30 (where that division loses precision) take a front-to-back phase
// instead, with SC_i, SD_i from totals recomputed in a first sweep.  The
// per-voxel gradients (8 corner densities, 3 colour channels) of all the
// warp's pixels are summed per staged entry in shared memory, and each entry
// that was hit is added to the global accumulators once per warp (a colour
// channel that the clamp of Eq. vox_color cut gets no gradient).
#include "svr_internal.cuh"

namespace svr {

constexpr int kWarps = 8;          // warps per CTA of the forward
constexpr int kThreads = kWarps * 32;
#ifndef SVR_FWD_MIN_BLOCKS
#define SVR_FWD_MIN_BLOCKS 3
#endif
constexpr int kFwdMinBlocks = SVR_FWD_MIN_BLOCKS;   // resident CTAs per SM the forward's register budget is sized for
constexpr int kBwdWarps = 4;       // warps per CTA of the backward (more shared memory per warp)
constexpr int kBwdThreads = kBwdWarps * 32;
#ifndef SVR_BWD_MIN_BLOCKS
#define SVR_BWD_MIN_BLOCKS 5
#endif
constexpr int kBwdMinBlocks = SVR_BWD_MIN_BLOCKS;   // resident CTAs per SM the register budget is sized for
constexpr int kBatch = 32;

// Staged list entry, padded to 112 bytes: lanes reading different entries
// then spread over 8 bank groups rather than 4.
struct Entry {
    float4 a;    // entry plane (near corner) relative to r_o, sign bits (int)
    float4 b;    // exit plane (far corner) relative to r_o, 1 / size
    float4 c;    // (min corner - r_o) / size, index in the sorted list (int)
    float4 g0;   // raw corner densities 0..3
    float4 g1;   // raw corner densities 4..7
    float4 col;  // colour, voxel id (int)
    float4 pad;  // x: clamp bits of the colour channels (uint); y, z, w unused
};

__device__ __forceinline__ void stage_entry(Entry &e, uint32_t val, int idx, const Record *__restrict__ rec) {
    const uint32_t s = val >> 29;
    const uint32_t vid = val & 0x1FFFFFFFu;
    const Record *r = rec + vid;
    const float4 r0 = __ldg(&r->r0);
    const float lx = r0.x, ly = r0.y, lz = r0.z, size = r0.w;
    const float hx = lx + size, hy = ly + size, hz = lz + size;
    const float inv = 1.0f / size;
    e.a = make_float4((s & 4) ? hx : lx, (s & 2) ? hy : ly, (s & 1) ? hz : lz, __int_as_float((int)s));
    e.b = make_float4((s & 4) ? lx : hx, (s & 2) ? ly : hy, (s & 1) ? lz : hz, inv);
    e.c = make_float4(lx * inv, ly * inv, lz * inv, __int_as_float(idx));
    e.g0 = __ldg(&r->r1);
    e.g1 = __ldg(&r->r2);
    const float4 c3 = __ldg(&r->r3);
    e.col = make_float4(c3.x, c3.y, c3.z, __int_as_float((int)vid));
    e.pad.x = c3.w;
}

// Trilinear interpolation of Eq. interp; corner bits (x, y, z), x most significant.
__device__ __forceinline__ float trilerp(const float4 &g0, const float4 &g1, float qx, float qy, float qz) {
    const float c00 = fmaf(qz, g0.y - g0.x, g0.x);  // 000, 001
    const float c01 = fmaf(qz, g0.w - g0.z, g0.z);  // 010, 011
    const float c10 = fmaf(qz, g1.y - g1.x, g1.x);  // 100, 101
    const float c11 = fmaf(qz, g1.w - g1.z, g1.z);  // 110, 111
    const float c0 = fmaf(qy, c01 - c00, c00);
    const float c1 = fmaf(qy, c11 - c10, c10);
    return fmaf(qx, c1 - c0, c0);
}

// alpha = 1 - exp(-X) of a segment with optical depth X = sum_k (l/K) sigma_k
// (Eq. supp_alpha_comp), given P = prod_k exp(-(l/K) sigma_k).  1 - P loses
// its relative precision as X -> 0 (P rounds to within 2^-24 of 1); below
// X = 1/32 the series X - X^2/2 + X^3/6 - X^4/24 is used instead, whose first
// omitted term is below 1e-8 of alpha there, so alpha (and every weight and
// gradient proportional to it) keeps its relative precision for faint voxels.
__device__ __forceinline__ float seg_alpha(float X, float P) {
    const float s = X * fmaf(-0.5f * X, fmaf(-0.333333333f * X, fmaf(-0.25f, X, 1.f), 1.f), 1.f);
    return X < 0.03125f ? s : 1.f - P;
}

struct PixelRay {
    float3 rd, inv;
    float rdn;
    int s;
    int x, y;
    bool inside;
};

struct WarpBlock {
    int x0, y0;      // origin of the warp's 8x4 pixel block
    unsigned smask;  // bit s set if one of its in-image pixels has sign bits s
    unsigned spix;   // lane t < 8: mask of the block's in-image pixels with sign bits t
};

// Per-view arrays of the work item's view.
struct ViewData {
    const Record *rec;    // f.rec + view * N
    const ushort4 *box;   // f.box + view * N
    DebugBlock *dbg;      // index checks of the SVR_DEBUG build
    int64_t n;            // N
};

// Voxel id of a list entry's value (index-checked in the SVR_DEBUG build).
__device__ __forceinline__ uint32_t vid_of(const ViewData &vd, uint32_t val) {
    return checked(vd.dbg, kDbgVoxel, val & 0x1FFFFFFFu, vd.n);
}

// Pixel of the calling lane in block blk of a tile (tile edge 8, 16 or 32:
// tile / 8 blocks of 8x4 pixels per block row).
__device__ __forceinline__ PixelRay pixel_ray(const DevCam &cam, int tile, int blk, WarpBlock &wb) {
    PixelRay p;
    const int tx = tile % cam.ntx, ty = tile / cam.ntx;
    const int lane = threadIdx.x & 31;
    const int bpr = cam.tile >> 3;
    wb.x0 = tx * cam.tile + (blk % bpr) * 8;
    wb.y0 = ty * cam.tile + (blk / bpr) * 4;
    p.x = wb.x0 + (lane & 7);
    p.y = wb.y0 + (lane >> 3);
    p.inside = p.x < cam.W && p.y < cam.H;
    p.rd = pixel_dir(cam, p.x, p.y);
    p.s = sign_bits(p.rd);
    // +0.0 for a zero component so that 1/r_d has the sign of the sign bits
    p.inv = make_float3(1.0f / (p.rd.x + 0.0f), 1.0f / (p.rd.y + 0.0f), 1.0f / (p.rd.z + 0.0f));
    p.rdn = sqrtf(p.rd.x * p.rd.x + p.rd.y * p.rd.y + p.rd.z * p.rd.z);
    wb.smask = __reduce_or_sync(0xffffffffu, p.inside ? (1u << p.s) : 0u);
    wb.spix = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const unsigned m = __ballot_sync(0xffffffffu, p.inside && p.s == t);
        if (lane == t) wb.spix = m;
    }
    return p;
}

// Mask of the block's pixels (bit 8 y + x) that may hit an entry: inside its
// inclusive pixel box bx and with its sign bits (value >> 29).  Called by all
// lanes; an invalid entry gives 0.
__device__ __forceinline__ unsigned entry_pixels(bool valid, uint32_t val, ushort4 bx, const WarpBlock &wb) {
    const unsigned spix = __shfl_sync(0xffffffffu, wb.spix, (int)(val >> 29));
    const int cx0 = max((int)bx.x - wb.x0, 0), cx1 = min((int)bx.y - wb.x0, 7);
    const int cy0 = max((int)bx.z - wb.y0, 0), cy1 = min((int)bx.w - wb.y0, 3);
    if (!valid || cx0 > cx1 || cy0 > cy1) return 0u;
    const unsigned row = (0xFFu << cx0) & (0xFFu >> (7 - cx1));
    const unsigned rows = (0xFFFFFFFFu << (8 * cy0)) & (0xFFFFFFFFu >> (8 * (3 - cy1)));
    return row * 0x01010101u & rows & spix;
}

// 32 x 32 bit-matrix transpose across the warp: lane i returns the word whose
// bit j is bit i of lane j's x (five exchanges of blocks of halving size).
__device__ __forceinline__ unsigned warp_transpose(unsigned x) {
    const int lane = threadIdx.x & 31;
    const unsigned masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int s = 16 >> i;
        const unsigned m = masks[i];
        const unsigned v = __shfl_xor_sync(0xffffffffu, x, s);
        x = (lane & s) ? ((x & ~m) | ((v & ~m) >> s)) : ((x & m) | ((v & m) << s));
    }
    return x;
}

// Slab test against a staged entry whose sign bits match the ray's.
__device__ __forceinline__ bool slab(const Entry &e, const PixelRay &p, float &a, float &b) {
    a = fmaxf(fmaxf(e.a.x * p.inv.x, e.a.y * p.inv.y), e.a.z * p.inv.z);
    b = fminf(fminf(e.b.x * p.inv.x, e.b.y * p.inv.y), e.b.z * p.inv.z);
    return a <= b && a > 0.f;
}

// ------------------------------------------------------------- block lists
//
// A warp renders one 8x4 block and needs only the entries of its tile's list
// whose pixel box meets the block and whose sign pattern a pixel of the block
// has.  k_block_lists extracts them once per frame, one CTA at a time per
// entry of the render work order (a tile, or one kSegLen-entry segment of a
// split tile):
// thread t loads entries t, t + kListThreads, ... of the segment (value and box) and
// writes each one's mask of such blocks to shared memory (the box's block
// rectangle AND the blocks holding a pixel with its sign bits, from the
// per-block sign masks of k_tile_mask); then warp w keeps the entries of
// blocks w, w + kListWarps, ... by ballot, which preserves list order, and writes
// (value, sorted index) pairs.  Block b of a tile whose list is [beg, end)
// owns the region B beg + b (end - beg) of the block lists, so the lists need
// no allocation scan; segment s of a split tile writes from offset s kSegLen
// of that region (it keeps at most kSegLen entries) and records its count per
// block.  The CTA of segment 0 also clears the tile's merge counters for the
// next forward.  The CTAs form a persistent grid that strides over the
// entries.

constexpr int kListThreads = 128;
constexpr int kListWarps = kListThreads / 32;
constexpr int kMaxBlocksPerWarp = 32 / kListWarps;  // tile 32: 32 blocks over the warps
constexpr int kListChunk = kSegLen;

__device__ __forceinline__ void block_lists_entry(const FrameDev &f, const uint32_t *__restrict__ vals, unsigned e,
                                                  uint32_t *sval, uint32_t *smsk) {
    const uint2 gs = f.order[e];
    const int g = (int)gs.x, sg = (int)gs.y;
    const int view = view_of_tile(f, g);
    const DevCam &cam = f.views[view];
    const int tile = g - cam.tile_base;
    const uint2 rg = f.ranges[g];
    if (!SVR_IN_BOUNDS(f.debug, kDbgRange, rg.y, f.capacity + 1)) return;
    const int beg = (int)rg.x, end = (int)rg.y, L = end - beg;
    const int B = f.blocks_per_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const ushort4 *boxes = f.box + (size_t)view * f.n_vox;
    const uint2 ts = f.tile_seg[g];
    const bool split = ts.x > 1;
    if (sg == 0 && threadIdx.x < B) f.merge_cnt[(size_t)g * B + threadIdx.x] = 0;
    // lane s < 8: mask of the tile's blocks with an in-image pixel of sign bits s
    const unsigned bsign = lane < B ? f.block_sign[(size_t)g * B + lane] : 0u;
    unsigned sblk = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const unsigned m = __ballot_sync(0xffffffffu, (bsign >> t) & 1u);
        if (lane == t) sblk = m;
    }
    const int T = cam.tile, bpr = T >> 3;
    const int tx0 = (tile % cam.ntx) * T, ty0 = (tile / cam.ntx) * T;
    // bit r bpr for each block row r: replicates a row's column bits over the rows
    const unsigned rep = bpr == 1 ? 0x3u : (bpr == 2 ? 0x55u : 0x11111111u);
    // a split tile's segment is one chunk; an unsplit list is walked whole
    const int first = beg + sg * kListChunk;
    const int stop = split ? min(end, first + kListChunk) : end;
    uint2 *out = f.blist + (size_t)B * beg + (split ? (size_t)sg * kListChunk : 0);
    unsigned cnt[kMaxBlocksPerWarp];
#pragma unroll
    for (int k = 0; k < kMaxBlocksPerWarp; ++k) cnt[k] = 0u;
    for (int c0 = first; c0 < stop; c0 += kListChunk) {
        const int n = min(kListChunk, stop - c0);
        uint32_t v4[kListChunk / kListThreads];
#pragma unroll
        for (int r = 0; r < kListChunk / kListThreads; ++r) {
            const int t = threadIdx.x + kListThreads * r;
            v4[r] = t < n ? __ldg(vals + c0 + t) : 0u;
        }
#pragma unroll
        for (int r = 0; r < kListChunk / kListThreads; ++r) {
            const int t = threadIdx.x + kListThreads * r;
            unsigned m = 0;
            if (t < n) {
                const ushort4 bx = __ldg(boxes + checked(f.debug, kDbgVoxel, v4[r] & 0x1FFFFFFFu, f.n_vox));
                const int cx0 = max((int)bx.x - tx0, 0), cx1 = min((int)bx.y - tx0, T - 1);
                const int cy0 = max((int)bx.z - ty0, 0), cy1 = min((int)bx.w - ty0, T - 1);
                if (cx0 <= cx1 && cy0 <= cy1) {
                    const unsigned cols = (2u << (cx1 >> 3)) - (1u << (cx0 >> 3));
                    const uint64_t rows = ((1ull << (((cy1 >> 2) + 1) * bpr)) - 1ull) &
                                          ~((1ull << ((cy0 >> 2) * bpr)) - 1ull);
                    m = cols * rep & (unsigned)rows;
                }
            }
            m &= __shfl_sync(0xffffffffu, sblk, (int)(v4[r] >> 29));
            if (t < n) {
                sval[t] = v4[r];
                smsk[t] = m;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kMaxBlocksPerWarp; ++k) {
            const int b = warp + kListWarps * k;
            if (b >= B) continue;
            for (int sub = 0; sub < n; sub += 32) {
                const int j = sub + lane;
                const bool keep = j < n && ((smsk[j] >> b) & 1u);
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) out[(size_t)b * L + cnt[k] + __popc(bal & lt)] = make_uint2(sval[j], (unsigned)(c0 + j));
                cnt[k] += __popc(bal);
            }
        }
        __syncthreads();
    }
    if (lane == 0) {
        uint32_t *len = split ? f.seg_len + (size_t)(ts.y + sg) * B : f.blen + (size_t)g * B;
#pragma unroll
        for (int k = 0; k < kMaxBlocksPerWarp; ++k)
            if (warp + kListWarps * k < B) len[warp + kListWarps * k] = cnt[k];
    }
}

// A persistent grid of CTAs takes the work-order entries in turn (the count
// is the device's).
__global__ void __launch_bounds__(kListThreads) k_block_lists(FrameDev f, const uint32_t *__restrict__ vals) {
    __shared__ uint32_t sval[kListChunk];
    __shared__ uint32_t smsk[kListChunk];
    const unsigned nq = f.status->n_listed;  // empty lists have no block lists
    for (unsigned e = blockIdx.x; e < nq; e += gridDim.x) {
        block_lists_entry(f, vals, e, sval, smsk);
        __syncthreads();  // shared memory is reused by the next entry
    }
}

// Exclusive prefix sum of v over the lanes of the warp; *total gets the sum.
__device__ __forceinline__ int warp_exclusive_scan(int v, int *total) {
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Software-pipelined walk of a block list: the next batch's (value, index)
// pair and pixel box are fetched while the current batch is staged and
// composited, so a batch waits on one dependent load (the record).
struct Lookahead {
    uint2 vi;   // value, sorted index
    ushort4 box;
    bool valid;
};

__device__ __forceinline__ void fetch_vi(Lookahead &la, const uint2 *__restrict__ list, int pos, bool valid) {
    la.valid = valid;
    la.vi = valid ? __ldg(list + pos) : make_uint2(0u, 0u);
}

__device__ __forceinline__ void fetch_box(Lookahead &la, const ViewData &vd) {
    la.box = la.valid ? __ldg(vd.box + vid_of(vd, la.vi.x)) : make_ushort4(0, 0, 0, 0);
}

// Ask for the looked-ahead entry's 64-byte record in L1 (the backward stages
// with plain loads one batch later).
__device__ __forceinline__ void prefetch_record(const Lookahead &la, const ViewData &vd) {
    if (la.valid) asm volatile("prefetch.global.L1 [%0];" ::"l"(vd.rec + vid_of(vd, la.vi.x)));
}

// Stage the looked-ahead entries (lane j: entry j of the batch).
__device__ __forceinline__ void stage_ahead(Entry *st, const ViewData &vd, const Lookahead &la) {
    if (la.valid) stage_entry(st[threadIdx.x & 31], (la.vi.x & 0xE0000000u) | vid_of(vd, la.vi.x), (int)la.vi.y, vd.rec);
    __syncwarp();
}

// First block-list position in [lo, hi) (entries sorted by index) whose
// index is at least key, found by the whole warp: each round the lanes probe
// the last entry of 32 equal chunks and keep the chunk holding the boundary,
// then one probe per position; a list up to 1024 entries long costs two
// dependent loads.
__device__ __forceinline__ int lower_pos(const uint2 *__restrict__ list, int lo, int hi, int key) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const int s = (hi - lo + 31) >> 5;       // chunk length
        const int pos = lo + (lane + 1) * s - 1;  // last position of chunk `lane`
        const bool below = pos < hi && (int)__ldg(&list[pos].y) < key;
        lo += s * __popc(__ballot_sync(0xffffffffu, below));  // chunks wholly below key
        hi = min(hi, lo + s);
    }
    const int pos = lo + lane;
    const bool below = pos < hi && (int)__ldg(&list[pos].y) < key;
    return lo + __popc(__ballot_sync(0xffffffffu, below));
}

// Work item of a render warp: segment `seg` of global tile g, 8x4 block blk.
struct Item {
    int g, seg, blk;
};

// Next work item of the calling warp, or false when done.
__device__ __forceinline__ bool next_item(unsigned *counter, unsigned n_items, unsigned blocks_per_tile,
                                          const uint2 *order, Item &it) {
    unsigned item = 0;
    if ((threadIdx.x & 31) == 0) item = atomicAdd(counter, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) return false;
    const uint2 q = order[item / blocks_per_tile];
    it.g = (int)q.x;
    it.seg = (int)q.y;
    it.blk = (int)(item % blocks_per_tile);
    return true;
}

// The view of a global tile and its arrays.
struct ItemView {
    int view;
    int tile;   // tile index within the view
    ViewData vd;
};

__device__ __forceinline__ ItemView item_view(const FrameDev &f, int g) {
    ItemView iv;
    iv.view = view_of_tile(f, g);
    iv.tile = g - f.views[iv.view].tile_base;
    iv.vd.rec = f.rec + (size_t)iv.view * f.n_vox;
    iv.vd.box = f.box + (size_t)iv.view * f.n_vox;
    iv.vd.dbg = f.debug;
    iv.vd.n = f.n_vox;
    return iv;
}

// The block list of an item and the part of it that its segment covers.
struct ItemList {
    const uint2 *list;  // the (tile, block) list
    int n_list;
    int beg, end;       // the tile's range in the sorted pairs
    uint2 ts;           // segments of the tile, first slot
    const uint32_t *seg_len; // split tiles: segment k of this block holds seg_len[k * B] entries
    DebugBlock *dbg;         // index checks of the SVR_DEBUG build
};

__device__ __forceinline__ ItemList item_list(const FrameDev &f, int g, int blk) {
    ItemList L;
    const uint2 rg = f.ranges[g];
    const int B = f.blocks_per_tile;
    L.beg = (int)rg.x;
    L.end = (int)rg.y;
    if (!SVR_IN_BOUNDS(f.debug, kDbgRange, rg.y, f.capacity + 1) || !SVR_IN_BOUNDS(f.debug, kDbgRange, rg.x, rg.y + 1))
        L.beg = L.end = 0;
    L.list = f.blist + (size_t)B * L.beg + (size_t)blk * (L.end - L.beg);
    // unsplit tiles (split ones count per segment); an empty tile's block
    // lengths are not written (k_block_lists skips empty lists)
    L.n_list = L.end > L.beg ? (int)f.blen[(size_t)g * B + blk] : 0;
    L.ts = f.tile_seg[g];
    if (L.ts.x <= 1 && !SVR_IN_BOUNDS(f.debug, kDbgBlockList, L.n_list, L.end - L.beg + 1)) L.n_list = 0;
    L.seg_len = f.seg_len + (size_t)L.ts.y * B + blk;
    L.dbg = f.debug;
    return L;
}

// Block-list positions [p0, p1) of segment sg of a split tile: segment sg
// owns the kSegLen positions from sg kSegLen.
__device__ __forceinline__ void seg_range(const ItemList &L, int B, int sg, int &p0, int &p1) {
    p0 = sg * kSegLen;
    p1 = p0 + (int)L.seg_len[(size_t)sg * B];
    if (!SVR_IN_BOUNDS(L.dbg, kDbgBlockList, p1 - p0, kSegLen + 1)) p1 = p0;
}

// The hit masks of an item's block list (see FrameDev::hmask): word p of the
// result belongs to block-list position p.  Only an item's first walk
// writes them (the merge's second walk of a segment and the max-weight pass
// leave them), so they hold every pixel's hits up to its stopping voxel.
__device__ __forceinline__ uint32_t *hit_masks(const FrameDev &f, const ItemList &L, const Item &it) {
    return f.hmask + (L.list - f.blist) + 32 * ((size_t)it.g * f.blocks_per_tile + it.blk);
}

// Segment sums of (segment slot, block): kSegFields rows of 32 pixels.
__device__ __forceinline__ float *seg_fields(const FrameDev &f, unsigned slot, int blk) {
    slot = checked(f.debug, kDbgSegSlot, slot, f.seg_slots);
    return f.seg_part + ((size_t)slot * f.blocks_per_tile + blk) * (kSegFields * 32) + (threadIdx.x & 31);
}

// ------------------------------------------------------------------ forward

// Local depth, transmittance factor and alpha of a hit.
template <int K>
__device__ __forceinline__ void hit_fwd(const Entry &e, const PixelRay &p, float a, float b, float &trans,
                                        float &dloc, float &alpha) {
    const float inv_k = 1.0f / K;
    const float seg = b - a;
    const float xs = seg * p.rdn * inv_k;
    const float step = seg * inv_k;
    const float inv_size = e.b.w;
    const float rx = p.rd.x * inv_size, ry = p.rd.y * inv_size, rz = p.rd.z * inv_size;
    float t = fmaf(0.5f, step, a);
    float P = 1.f, d = 0.f, X = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float v = trilerp(e.g0, e.g1, fmaf(t, rx, -e.c.x), fmaf(t, ry, -e.c.y), fmaf(t, rz, -e.c.z));
        const float xk = xs * explin(v);
        const float ek = __expf(-xk);
        d = fmaf(P * (1.f - ek), t, d);
        P *= ek;
        X += xk;
        t += step;
    }
    trans = P;
    dloc = d;
    alpha = seg_alpha(X, P);
}

struct FwdOut {
    float *rgb, *depth, *alpha, *T;
    int32_t *last;
    int2 *stats;
    float *normal;      // extras: [3][H][W] composited voxel normals, or NULL
    float *max_weight;  // extras: [N] per-voxel maximum of T_i alpha_i, raised with atomicMax, or NULL
    float *dist;        // extras: [2][H][W] distortion loss of each ray and sum_i w_i m_i, or NULL
};

// Forward variants: the plain render, the work-counting one, and the one with
// the extra outputs (normal image, maximum blending weights).
constexpr int kModePlain = 0, kModeStats = 1, kModeExtra = 2, kModeDist = 3;

// Compositing state of the calling lane's pixel.
struct FwdState {
    float T, C0, C1, C2, D;
    int last;     // sorted index of the voxel that stopped the walk, or -1
    bool done;
    int n_cand, n_hit;
    float N0, N1, N2;  // composited normal (extras)
    // distortion loss (extras): the loss so far, and the sums of the weights
    // w_i = T_i alpha_i and of w_i m_i (m_i the segment's midpoint) so far
    float LD, PW, PS;
};

// Distortion loss (Sec. 3.2.3, the loss of Mip-NeRF 360) over a ray's
// composited voxels, with weights w_i, interval midpoints m_i = (a_i + b_i) / 2
// and lengths delta_i = b_i - a_i in ray distance:
//   L = sum_i sum_j w_i w_j |m_i - m_j| + 1/3 sum_i w_i^2 delta_i.
// Front to back (the voxels' intervals do not overlap, so m grows along the
// list) each voxel adds 2 w_i (m_i W_<i - S_<i) + w_i^2 delta_i / 3 with the
// prefix sums W_<i = sum_{j<i} w_j, S_<i = sum_{j<i} w_j m_j.
__device__ __forceinline__ void dist_add(FwdState &s, float w, float a, float b) {
    const float m = 0.5f * (a + b);
    s.LD += fmaf(2.f * w, fmaf(m, s.PW, -s.PS), w * w * (b - a) * 0.333333333f);
    s.PW += w;
    s.PS = fmaf(w, m, s.PS);
}

// Voxel normal of Eq. vox_normal from the 8 raw corner densities (corner c:
// bit 2 = x, bit 1 = y, bit 0 = z; g0 = corners 0..3, g1 = 4..7): the
// gradient of the trilinear field at the centre, Eq. interp_grad (a quarter
// of far face minus near face per axis; the factor cancels here), normalised;
// zero where the gradient vanishes.  Returns the gradient's length (of the
// unscaled differences times 1/4).
__device__ __forceinline__ float voxel_normal(const float4 &g0, const float4 &g1, float3 &n) {
    const float gx = 0.25f * ((g1.x + g1.y + g1.z + g1.w) - (g0.x + g0.y + g0.z + g0.w));
    const float gy = 0.25f * ((g0.z + g0.w + g1.z + g1.w) - (g0.x + g0.y + g1.x + g1.y));
    const float gz = 0.25f * ((g0.y + g0.w + g1.y + g1.w) - (g0.x + g0.z + g1.x + g1.z));
    const float len = sqrtf(gx * gx + gy * gy + gz * gz);
    const float inv = len > 0.f ? 1.0f / len : 0.f;
    n = make_float3(gx * inv, gy * inv, gz * inv);
    return len;
}

// Asynchronous staging of the forward.  A slot receives a voxel's 64-byte
// record as copied (cp.async, 16 bytes per copy, no registers involved);
// once the copy has landed, lane j turns the first part (min corner, size)
// of its slot into the entry plane and 1 / size and writes the exit plane,
// both from the entry's sign bits.  Slots are 80 bytes apart, which spreads
// lanes reading different slots over the shared-memory banks.
struct FwdSlot {
    float4 a;    // copied: min corner relative to r_o, size; then: entry plane, 1 / size
    float4 g0;   // raw corner densities 0..3
    float4 g1;   // raw corner densities 4..7
    float4 col;  // colour, clamp bits
    float4 b;    // exit plane
};

// Hits of one batch handed to the lanes at a time by the hit-parallel
// compositing (phase B of the plain and counting forwards).
#ifndef SVR_FWD_HIT_CAP
#define SVR_FWD_HIT_CAP 128
#endif
constexpr int kHitCap = SVR_FWD_HIT_CAP;
// The hit-parallel pass is taken when kHpNum * (busiest pixel's hits) >
// kHpDen * (rounds of 32 hits); measured on the 1M-voxel frame over 1/1,
// 2/3, 1/2, 1/3 and never: 1/2 is fastest (0.205 vs 0.215 ms never, 0.244
// always).  Overridable at build time for such sweeps.
#ifndef SVR_FWD_HP_NUM
#define SVR_FWD_HP_NUM 1
#define SVR_FWD_HP_DEN 2
#endif
constexpr int kHpNum = SVR_FWD_HP_NUM, kHpDen = SVR_FWD_HP_DEN;

struct FwdSmem {
    FwdSlot slot[2][kBatch];  // double buffer: the batch being composited and the next one
    uint2 meta[2][kBatch];    // (value, sorted index) of each staged entry
    float4 hres[kHitCap];     // per hit: transmittance factor, alpha, local depth
    uint16_t hpair[kHitCap];  // per hit: pixel lane << 5 | staged entry
};

// Lane j starts the copy of its entry's record into buffer buf; every lane
// commits a group (possibly empty) so that the group counts stay aligned.
__device__ __forceinline__ void stage_async(FwdSmem &ws, int buf, const ViewData &vd, const Lookahead &la) {
    const int lane = threadIdx.x & 31;
    if (la.valid) {
        const Record *r = vd.rec + vid_of(vd, la.vi.x);
        FwdSlot &d = ws.slot[buf][lane];
        cp_async16(&d.a, &r->r0);
        cp_async16(&d.g0, &r->r1);
        cp_async16(&d.g1, &r->r2);
        cp_async16(&d.col, &r->r3);
        ws.meta[buf][lane] = la.vi;
    }
    cp_async_commit();
}

// Entry and exit planes of lane j's staged record (copied: min corner, size)
// from the entry's sign bits s: the near corner is min + size on the axes
// where r_d is negative.
__device__ __forceinline__ void slot_planes(FwdSlot &d, uint32_t s) {
    const float4 r0 = d.a;
    const float hx = r0.x + r0.w, hy = r0.y + r0.w, hz = r0.z + r0.w;
    d.a = make_float4((s & 4) ? hx : r0.x, (s & 2) ? hy : r0.y, (s & 1) ? hz : r0.z, 1.0f / r0.w);
    d.b = make_float4((s & 4) ? r0.x : hx, (s & 2) ? r0.y : hy, (s & 1) ? r0.z : hz, 0.f);
}

__device__ __forceinline__ bool slab_slot(const FwdSlot &e, const PixelRay &p, float &a, float &b) {
    const float4 ea = e.a, eb = e.b;
    a = fmaxf(fmaxf(ea.x * p.inv.x, ea.y * p.inv.y), ea.z * p.inv.z);
    b = fminf(fminf(eb.x * p.inv.x, eb.y * p.inv.y), eb.z * p.inv.z);
    return a <= b && a > 0.f;
}

// Local depth and transmittance factor of a hit on a staged slot (its sign
// bits are the pixel's, sb = 1 where r_d is negative: the min corner is the
// exit plane there and the entry plane elsewhere).
template <int K>
__device__ __forceinline__ void hit_fwd_slot(const FwdSlot &e, const PixelRay &p, const float3 &sb, float a,
                                             float b, float &trans, float &dloc, float &alpha) {
    const float inv_k = 1.0f / K;
    const float seg = b - a;
    const float xs = seg * p.rdn * inv_k;
    const float step = seg * inv_k;
    const float4 ea = e.a, eb = e.b;
    const float inv = ea.w;
    const float cx = (sb.x != 0.f ? eb.x : ea.x) * inv, cy = (sb.y != 0.f ? eb.y : ea.y) * inv,
                cz = (sb.z != 0.f ? eb.z : ea.z) * inv;
    const float4 g0 = e.g0, g1 = e.g1;
    const float rx = p.rd.x * inv, ry = p.rd.y * inv, rz = p.rd.z * inv;
    float t = fmaf(0.5f, step, a);
    float P = 1.f, d = 0.f, X = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float v = trilerp(g0, g1, fmaf(t, rx, -cx), fmaf(t, ry, -cy), fmaf(t, rz, -cz));
        const float xk = xs * explin(v);
        const float ek = __expf(-xk);
        d = fmaf(P * (1.f - ek), t, d);
        P *= ek;
        X += xk;
        t += step;
    }
    trans = P;
    dloc = d;
    alpha = seg_alpha(X, P);
}

// Phase B of a batch, hit-parallel: the batch's (pixel, entry) hits are
// listed pixel by pixel, in list order within a pixel, and handed to the
// lanes kHitCap at a time; lane t takes hit t whatever its pixel (the
// pixel's ray comes by shuffle) and computes the costly part, its
// transmittance factor, alpha and local depth (K trilinear samples and
// exponentials), into the warp's hit buffer; then every pixel composites its
// own hits from the buffer in list order, a few multiply-adds each, and stops
// once T < t_stop.  So the lanes do the per-hit arithmetic together however
// unevenly the hits fall on the pixels.
template <int K, bool STATS>
__device__ __forceinline__ void fwd_hits_parallel(const FwdSlot *st, const uint2 *meta, FwdSmem &ws,
                                                  const PixelRay &p, const float3 &sb, unsigned hits, float t_stop,
                                                  FwdState &s) {
    const int lane = threadIdx.x & 31;
    int total;
    const int off = warp_exclusive_scan(__popc(hits), &total);
    for (int h0 = 0; h0 < total; h0 += kHitCap) {
        const int hn = min(kHitCap, total - h0);
        // list this chunk's hits: lane l's i-th hit is hit off_l + i
        {
            unsigned h = hits;
            for (int i = off; h; ++i, h &= h - 1u)
                if (i >= h0 && i < h0 + hn) ws.hpair[i - h0] = (uint16_t)((lane << 5) | (__ffs(h) - 1));
        }
        __syncwarp();
        for (int r = 0; r < hn; r += 32) {
            const int t = r + lane;
            const unsigned pr = t < hn ? ws.hpair[t] : (unsigned)(lane << 5);
            const int l = (int)(pr >> 5);
            PixelRay q;
            q.rd = make_float3(__shfl_sync(0xffffffffu, p.rd.x, l), __shfl_sync(0xffffffffu, p.rd.y, l),
                               __shfl_sync(0xffffffffu, p.rd.z, l));
            q.inv = make_float3(__shfl_sync(0xffffffffu, p.inv.x, l), __shfl_sync(0xffffffffu, p.inv.y, l),
                                __shfl_sync(0xffffffffu, p.inv.z, l));
            q.rdn = __shfl_sync(0xffffffffu, p.rdn, l);
            const float3 qsb = make_float3(__shfl_sync(0xffffffffu, sb.x, l), __shfl_sync(0xffffffffu, sb.y, l),
                                           __shfl_sync(0xffffffffu, sb.z, l));
            if (t < hn) {
                const FwdSlot &e = st[pr & 31u];
                float a, b;
                slab_slot(e, q, a, b);
                float P, dloc, al;
                hit_fwd_slot<K>(e, q, qsb, a, b, P, dloc, al);
                ws.hres[t] = make_float4(P, al, dloc, 0.f);
            }
        }
        __syncwarp();
        // each pixel composites its hits of this chunk in order
        const int i0 = max(off, h0), i1 = min(off + __popc(hits), h0 + hn);
        if (!s.done) {
            for (int i = i0; i < i1; ++i) {
                const int t = i - h0;
                const float4 hr = ws.hres[t];
                const int k = ws.hpair[t] & 31;
                const float4 col = st[k].col;
                const float w = s.T * hr.y;
                s.C0 = fmaf(w, col.x, s.C0);
                s.C1 = fmaf(w, col.y, s.C1);
                s.C2 = fmaf(w, col.z, s.C2);
                s.D = fmaf(s.T, hr.z, s.D);
                s.T *= hr.x;
                if (STATS) ++s.n_hit;
                if (s.T < t_stop) {
                    s.done = true;
                    s.last = (int)meta[k].y;
                    break;
                }
            }
        }
        __syncwarp();
    }
}

// Walk block-list positions [p0, p1) front to back from state s.  The list
// entries are fetched two batches ahead and the next batch's records are
// copied into the other staging buffer while this batch is composited.
template <int K, int MODE>
__device__ __forceinline__ void fwd_walk(const uint2 *__restrict__ list, int p0, int p1, const ViewData &vd,
                                         const PixelRay &p, const WarpBlock &wb, FwdSmem &ws, float t_stop,
                                         FwdState &s, const FwdOut &out, bool true_weights, uint32_t *hm) {
    constexpr bool STATS = MODE == kModeStats, FN = MODE == kModeExtra, FD = FN || MODE == kModeDist;
    constexpr bool EXTRA = FN || FD;
    const int lane = threadIdx.x & 31;
    const float3 sb = make_float3((p.s & 4) ? 1.f : 0.f, (p.s & 2) ? 1.f : 0.f, (p.s & 1) ? 1.f : 0.f);
    Lookahead cur, nx, nn;
    fetch_vi(cur, list, p0 + lane, p0 + lane < p1);
    fetch_box(cur, vd);
    stage_async(ws, 0, vd, cur);
    fetch_vi(nx, list, p0 + kBatch + lane, p0 + kBatch + lane < p1);
    int buf = 0;
    for (int base = p0; base < p1; base += kBatch, buf ^= 1) {
        if (__all_sync(0xffffffffu, s.done)) break;
        fetch_box(nx, vd);
        stage_async(ws, buf ^ 1, vd, nx);
        const int npos = base + 2 * kBatch + lane;
        fetch_vi(nn, list, npos, npos < p1);
        const unsigned cand = warp_transpose(entry_pixels(cur.valid, cur.vi.x, cur.box, wb));
        cp_async_wait<1>();  // this batch's copies (the next batch's may still be in flight)
        __syncwarp();
        if (cur.valid) slot_planes(ws.slot[buf][lane], cur.vi.x >> 29);
        __syncwarp();
        const FwdSlot *st = ws.slot[buf];
        // phase A: this pixel's hits among its candidate entries
        unsigned hits = 0;
        if (!s.done) {
            for (unsigned c = cand; c; c &= c - 1u) {
                const int k = __ffs(c) - 1;
                if (STATS) ++s.n_cand;
                float a, b;
                if (slab_slot(st[k], p, a, b)) hits |= 1u << k;
            }
        }
        // this pixel's hits in the batch, for the backward
        if (hm != nullptr) hm[base + lane] = hits;
        if constexpr (!EXTRA) {
            // hit-parallel when the hits fall unevenly enough on the pixels:
            // the per-pixel rounds cost the busiest pixel's hit count, the
            // hit-parallel pass kHpDen / kHpNum rounds per 32 hits
            const int nh = __popc(hits);
            const int maxh = __reduce_max_sync(0xffffffffu, (unsigned)nh);
            const int tot = __reduce_add_sync(0xffffffffu, (unsigned)nh);
            if (kHpNum * maxh > kHpDen * ((tot + 31) >> 5)) {
                fwd_hits_parallel<K, STATS>(st, ws.meta[buf], ws, p, sb, hits, t_stop, s);
                __syncwarp();
                cur = nx;
                nx = nn;
                continue;
            }
        }
        // phase B: composite them in list order, one hit per pixel per round
        while (__any_sync(0xffffffffu, hits != 0)) {
            if (hits != 0) {
                const int k = __ffs(hits) - 1;
                hits &= hits - 1;
                const FwdSlot &e = st[k];
                float a, b;
                slab_slot(e, p, a, b);
                if (STATS) ++s.n_hit;
                float P, dloc, al;
                hit_fwd_slot<K>(e, p, sb, a, b, P, dloc, al);
                const float4 col = e.col;
                const float w = s.T * al;
                s.C0 = fmaf(w, col.x, s.C0);
                s.C1 = fmaf(w, col.y, s.C1);
                s.C2 = fmaf(w, col.z, s.C2);
                s.D = fmaf(s.T, dloc, s.D);
                if (EXTRA) {
                    if (FN && out.normal) {
                        float3 n;
                        voxel_normal(e.g0, e.g1, n);
                        s.N0 = fmaf(w, n.x, s.N0);
                        s.N1 = fmaf(w, n.y, s.N1);
                        s.N2 = fmaf(w, n.z, s.N2);
                    }
                    if (FD && out.dist) dist_add(s, w, a, b);
                    // weights are exact only when the walk started from the
                    // true transmittance (not a split segment's T = 1)
                    if (FN && out.max_weight && true_weights)
                        atomicMax(reinterpret_cast<int *>(out.max_weight) + vid_of(vd, ws.meta[buf][k].x),
                                  __float_as_int(w));
                }
                s.T *= P;
                if (s.T < t_stop) {
                    s.done = true;
                    s.last = (int)ws.meta[buf][k].y;
                    hits = 0;
                }
            }
        }
        __syncwarp();
        cur = nx;
        nx = nn;
    }
    cp_async_wait<0>();  // no copy may land in a buffer after the walk
    __syncwarp();
}

// Merge the segments of a split tile's block, front to back: segment sg was
// walked from T = 1, so its pixel adds T_before (C_sg, D_sg) and multiplies
// T by T_sg, unless the product falls below t_stop: then the pixel stopped
// inside sg (segment 0 already stopped at the right voxel; a later one is
// walked again from the merged state to find it).  Leaves per segment, for
// the backward: the transmittance after and before it and the colour and
// depth sums behind it (T_final bg included).
template <int K, int MODE>
__device__ __forceinline__ void fwd_merge(const FrameDev &f, const ItemList &L, int blk, const ViewData &vd,
                                          const PixelRay &p, const WarpBlock &wb, FwdSmem &ws, FwdState &m,
                                          const FwdOut &out) {
    constexpr bool STATS = MODE == kModeStats, FN = MODE == kModeExtra, FD = FN || MODE == kModeDist;
    const int B = f.blocks_per_tile;
    const int nseg = (int)L.ts.x;
    for (int sg = 0; sg < nseg; ++sg) {
        float *q = seg_fields(f, L.ts.y + sg, blk);
        const float Tb = m.T;
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, dd = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
        // distortion: the segment's internal loss and its sums of w, w m
        float dl_b = 0.f, dw_b = 0.f, ds_b = 0.f;
        const float W_before = m.PW, S_before = m.PS, L_before = m.LD;
        bool need = false;
        if (!m.done) {
            const float Tl = __ldcg(q + 4 * 32);
            if (Tb * Tl >= f.t_stop || sg == 0) {
                c0 = Tb * __ldcg(q);
                c1 = Tb * __ldcg(q + 32);
                c2 = Tb * __ldcg(q + 2 * 32);
                dd = Tb * __ldcg(q + 3 * 32);
                if (FN) {
                    n0 = Tb * __ldcg(q + 8 * 32);
                    n1 = Tb * __ldcg(q + 9 * 32);
                    n2 = Tb * __ldcg(q + 10 * 32);
                }
                if (FD) {
                    // segment walked from T = 1: its weights scale by Tb
                    dl_b = Tb * Tb * __ldcg(q + 11 * 32);
                    dw_b = Tb * __ldcg(q + 12 * 32);
                    ds_b = Tb * __ldcg(q + 13 * 32);
                }
                m.T = Tb * Tl;
                if (Tb * Tl < f.t_stop) {  // segment 0 stopped by itself
                    m.done = true;
                    m.last = __float_as_int(__ldcg(q + 5 * 32));
                }
                if (STATS) {
                    m.n_cand += __float_as_int(__ldcg(q + 6 * 32));
                    m.n_hit += __float_as_int(__ldcg(q + 7 * 32));
                }
            } else {
                need = true;
            }
        }
        if (__any_sync(0xffffffffu, need)) {
            FwdState r = {Tb, 0.f, 0.f, 0.f, 0.f, -1, !need, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            int p0, p1;
            seg_range(L, B, sg, p0, p1);
            fwd_walk<K, MODE>(L.list, p0, p1, vd, p, wb, ws, f.t_stop, r, out, true, nullptr);
            if (need) {
                c0 = r.C0;
                c1 = r.C1;
                c2 = r.C2;
                dd = r.D;
                n0 = r.N0;
                n1 = r.N1;
                n2 = r.N2;
                dl_b = r.LD;
                dw_b = r.PW;
                ds_b = r.PS;
                m.T = r.T;
                if (r.done) {
                    m.done = true;
                    m.last = r.last;
                }
                m.n_cand += r.n_cand;
                m.n_hit += r.n_hit;
            }
        }
        m.C0 += c0;
        m.C1 += c1;
        m.C2 += c2;
        m.D += dd;
        q[0] = c0;
        q[32] = c1;
        q[2 * 32] = c2;
        q[3 * 32] = dd;
        q[4 * 32] = m.T;
        q[5 * 32] = Tb;
        if (FN) {
            m.N0 += n0;
            m.N1 += n1;
            m.N2 += n2;
            q[8 * 32] = n0;
            q[9 * 32] = n1;
            q[10 * 32] = n2;
        }
        if (FD) {
            // the segment's pairs with the voxels before it
            m.LD = L_before + dl_b + 2.f * (ds_b * W_before - dw_b * S_before);
            m.PW = W_before + dw_b;
            m.PS = S_before + ds_b;
            q[11 * 32] = dl_b;
            q[12 * 32] = dw_b;
            q[13 * 32] = ds_b;
        }
    }
    // sums behind each segment, back to front; for the distortion loss the
    // weight sums behind it and sum_{j behind} w_j dL/dw_j, where a segment B
    // with A in front and C behind contributes 2 L_B + 2 (S_B W_A - W_B S_A)
    // + 2 (W_B S_C - S_B W_C) (L_B its internal loss, W, S the sums of w, w m)
    float S0 = m.T * f.bg[0], S1 = m.T * f.bg[1], S2 = m.T * f.bg[2], SD = 0.f, SN0 = 0.f, SN1 = 0.f, SN2 = 0.f;
    float WC = 0.f, SCc = 0.f, RWC = 0.f;
    const float W_tot = m.PW, S_tot = m.PS;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        float *q = seg_fields(f, L.ts.y + sg, blk);
        const float c0 = q[0], c1 = q[32], c2 = q[2 * 32], dd = q[3 * 32];
        q[0] = S0;
        q[32] = S1;
        q[2 * 32] = S2;
        q[3 * 32] = SD;
        S0 += c0;
        S1 += c1;
        S2 += c2;
        SD += dd;
        if (FN) {
            const float n0 = q[8 * 32], n1 = q[9 * 32], n2 = q[10 * 32];
            q[8 * 32] = SN0;
            q[9 * 32] = SN1;
            q[10 * 32] = SN2;
            SN0 += n0;
            SN1 += n1;
            SN2 += n2;
        }
        if (FD) {
            const float dl_b = q[11 * 32], dw_b = q[12 * 32], ds_b = q[13 * 32];
            const float WA = W_tot - WC - dw_b, SA = S_tot - SCc - ds_b;
            q[11 * 32] = WC;
            q[12 * 32] = SCc;
            q[13 * 32] = RWC;
            RWC += 2.f * dl_b + 2.f * (ds_b * WA - dw_b * SA) + 2.f * (dw_b * SCc - ds_b * WC);
            WC += dw_b;
            SCc += ds_b;
        }
    }
}

template <int MODE>
__device__ __forceinline__ void fwd_write(const FrameDev &f, const DevCam &cam, const PixelRay &p,
                                          const FwdState &s, int last, const FwdOut &out) {
    constexpr bool STATS = MODE == kModeStats, FN = MODE == kModeExtra, FD = FN || MODE == kModeDist;
    if (!p.inside) return;
    // outputs of view v start at pixel pix_base (rgb: 3 * pix_base, planar)
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t px = (size_t)p.y * cam.W + p.x;
    const size_t o = (size_t)cam.pix_base + px;
    float *rgb = out.rgb + 3 * (size_t)cam.pix_base + px;
    rgb[0] = fmaf(s.T, f.bg[0], s.C0);
    rgb[HW] = fmaf(s.T, f.bg[1], s.C1);
    rgb[2 * HW] = fmaf(s.T, f.bg[2], s.C2);
    out.depth[o] = s.D;
    out.alpha[o] = 1.f - s.T;
    out.T[o] = s.T;
    out.last[o] = last;
    if (STATS) out.stats[o] = make_int2(s.n_cand, s.n_hit);
    if (FN && out.normal) {
        float *nrm = out.normal + 3 * (size_t)cam.pix_base + px;
        nrm[0] = s.N0;
        nrm[HW] = s.N1;
        nrm[2 * HW] = s.N2;
    }
    if (FD && out.dist) {
        float *dst = out.dist + 2 * (size_t)cam.pix_base + px;
        dst[0] = s.LD;
        dst[HW] = s.PS;
    }
}

template <int K, int MODE>
__device__ __forceinline__ void fwd_item(const FrameDev &f, const Item &it, FwdSmem &ws, const FwdOut &out) {
    constexpr bool STATS = MODE == kModeStats, FN = MODE == kModeExtra, FD = FN || MODE == kModeDist;
    const ItemView iv = item_view(f, it.g);
    const DevCam &cam = f.views[iv.view];
    WarpBlock wb;
    const PixelRay p = pixel_ray(cam, iv.tile, it.blk, wb);
    if (wb.smask == 0) return;  // the whole block lies outside the image
    const ItemList L = item_list(f, it.g, it.blk);
    const int lane = threadIdx.x & 31;
    FwdState s = {1.f, 0.f, 0.f, 0.f, 0.f, -1, !p.inside, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (L.ts.x <= 1) {
        fwd_walk<K, MODE>(L.list, 0, L.n_list, iv.vd, p, wb, ws, f.t_stop, s, out, true, hit_masks(f, L, it));
        fwd_write<MODE>(f, cam, p, s, s.last >= 0 ? s.last : L.end - 1, out);
        return;
    }
    // one segment of a split tile, walked from T = 1
    const int B = f.blocks_per_tile;
    int p0, p1;
    seg_range(L, B, it.seg, p0, p1);
    fwd_walk<K, MODE>(L.list, p0, p1, iv.vd, p, wb, ws, f.t_stop, s, out, it.seg == 0, hit_masks(f, L, it));
    float *q = seg_fields(f, L.ts.y + it.seg, it.blk);
    q[0] = s.C0;
    q[32] = s.C1;
    q[2 * 32] = s.C2;
    q[3 * 32] = s.D;
    q[4 * 32] = s.T;
    q[5 * 32] = __int_as_float(s.last);
    if (STATS) {
        q[6 * 32] = __int_as_float(s.n_cand);
        q[7 * 32] = __int_as_float(s.n_hit);
    }
    if (FN) {
        q[8 * 32] = s.N0;
        q[9 * 32] = s.N1;
        q[10 * 32] = s.N2;
    }
    if (FD) {
        q[11 * 32] = s.LD;
        q[12 * 32] = s.PW;
        q[13 * 32] = s.PS;
    }
    __threadfence();
    __syncwarp();
    unsigned prev = 0;
    unsigned *cnt = f.merge_cnt + (size_t)it.g * B + it.blk;
    if (lane == 0) prev = atomicAdd(cnt, 1u);
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev + 1 != L.ts.x) return;
    // the last segment of the block to finish merges them all
    __threadfence();
    FwdState m = {1.f, 0.f, 0.f, 0.f, 0.f, -1, !p.inside, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    fwd_merge<K, MODE>(f, L, it.blk, iv.vd, p, wb, ws, m, out);
    fwd_write<MODE>(f, cam, p, m, m.last >= 0 ? m.last : L.end - 1, out);
    if (lane == 0) *cnt = 0;  // ready for the next forward of this sort
}

// MODE kModeStats: also count, per pixel, the list entries with its sign
// bits whose pixel box contains it (the slab tests it must make) and the hits
// it composited (int2 per pixel), for work accounting.  kModeExtra: the
// normal image, the per-voxel maximum blending weights and the distortion
// loss (whichever of out.normal, out.max_weight, out.dist is set).
// kModeDist: the distortion loss alone (the training step's extra).
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads, kFwdMinBlocks) k_render_fwd(FrameDev f, FwdOut out) {
    __shared__ FwdSmem smem[kWarps];
    FwdSmem &ws = smem[threadIdx.x >> 5];
    const unsigned bpt = (unsigned)f.blocks_per_tile;
    const unsigned n_items = f.status->n_queue * bpt;
    Item it;
    while (next_item(&f.status->fwd_next, n_items, bpt, f.order, it)) {
        fwd_item<K, MODE>(f, it, ws, out);
        __syncwarp();
    }
    // the launch's last warp to run out of work resets the work counter for
    // the next launch and marks the segment sums as this sort's
    if ((threadIdx.x & 31) == 0) {
        __threadfence();
        if (atomicAdd(&f.status->fwd_exit, 1u) == gridDim.x * (blockDim.x >> 5) - 1) {
            f.status->fwd_next = 0;
            f.status->fwd_exit = 0;
            // bit 1: the segment sums include the normal image, bit 2: the
            // distortion sums
            f.status->fwd_done = 1u | ((MODE == kModeExtra && out.normal) ? 2u : 0u) |
                                 (((MODE == kModeExtra || MODE == kModeDist) && out.dist) ? 4u : 0u);
        }
    }
}

// Maximum blending weights of the later segments of split tile lists (the
// forward's segment walks start from T = 1, so only segment 0 records its
// weights there): every such (segment, block) item is walked again from the
// transmittance that the forward's merge left in front of it, in parallel
// over the items, so each weight is the true T_i alpha_i.
template <int K>
__global__ void __launch_bounds__(kThreads, kFwdMinBlocks) k_render_maxw(FrameDev f, FwdOut out) {
    __shared__ FwdSmem smem[kWarps];
    FwdSmem &ws = smem[threadIdx.x >> 5];
    const unsigned bpt = (unsigned)f.blocks_per_tile;
    const unsigned n_items = f.status->n_listed * bpt;  // split tiles are among the listed
    Item it;
    while (next_item(&f.status->maxw_next, n_items, bpt, f.order, it)) {
        if (it.seg == 0) continue;
        const ItemView iv = item_view(f, it.g);
        const DevCam &cam = f.views[iv.view];
        WarpBlock wb;
        const PixelRay p = pixel_ray(cam, iv.tile, it.blk, wb);
        if (wb.smask == 0) continue;
        const ItemList L = item_list(f, it.g, it.blk);
        if (L.ts.x <= 1) continue;
        const float Tb = __ldcg(seg_fields(f, L.ts.y + it.seg, it.blk) + 5 * 32);
        FwdState s = {Tb, 0.f, 0.f, 0.f, 0.f, -1, !p.inside || !(Tb >= f.t_stop), 0, 0,
                      0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int p0, p1;
        seg_range(L, f.blocks_per_tile, it.seg, p0, p1);
        fwd_walk<K, kModeExtra>(L.list, p0, p1, iv.vd, p, wb, ws, f.t_stop, s, out, true, nullptr);
        __syncwarp();
    }
}

// ----------------------------------------------------------------- backward

struct PixelGrad {
    float gC0, gC1, gC2, gD, gA;
    float Tfin;
    float gN0, gN1, gN2;  // upstream gradient of the normal image (extras)
    float gL;             // upstream gradient of the ray's distortion loss (extras)
    float Wtot, Stot;     // its totals sum w_i = 1 - T_final and sum w_i m_i
};

// Distortion sums behind a voxel: of w_j, of w_j m_j and of w_j dL/dw_j.
struct DistSums {
    float W, S, R;
};

// Sums of the normal image behind a voxel (extras; like SC for colour).
struct NrmSums {
    float x, y, z;
};

// Backward extras selected at compile time (XM bits): the normal image's
// gradient, the distortion loss's gradient, the pruning/subdivision statistics
// (priority and max weight).  Instantiated for none, distortion, distortion
// with the statistics, and all.
constexpr int kXNrm = 1, kXDist = 2, kXStat = 4, kXAll = 7;

// Gradient contributions of one hit, computed from one pass over its K
// samples.  B2F: T_known is the transmittance behind the voxel (T_{i+1}) and
// SC, SD the sums strictly behind it.  Front to back: T_known is T_i and
// SC, SD are the sums behind AND including the voxel (total minus the
// prefix before it); the voxel's own share is removed here.  Returns the
// transmittance in front of the voxel (T_i) and behind it (T_{i+1}), its
// blending weight and local depth.
// kXNrm: the normal image joins the objective (SN: its sums behind the voxel,
// like SC; nrm returns the voxel's normal).  kXStat: prio returns the voxel's
// subdivision priority term |alpha dL/dalpha| (Eq. priority), alpha dL/dalpha
// = alpha / (1 - alpha) dL/dx with x the optical depth.
// kXDist, with the distortion loss (g.gL != 0): dL/dw_i = 2 (m_i W_<i - S_<i) +
// 2 (S_>i - m_i W_>i) + 2/3 w_i delta_i (returned in cdist, prefix sums as the
// totals minus the sums behind, DS, and the voxel's own), and it joins dL/dx_i
// like a colour: T_(i+1) dL/dw_i - sum_{j>i} w_j dL/dw_j.
template <int K, bool B2F, int XM>
__device__ __forceinline__ void hit_grad(const Entry &e, const PixelRay &p, const PixelGrad &g, float a, float b,
                                         float T_known, float SC0, float SC1, float SC2, float SD, NrmSums SN,
                                         DistSums DS, float dgeo[8], float dcol[3], float &T_i, float &T_after,
                                         float &w, float &dloc, float3 &nrm, float &prio, float &cdist) {
    const float inv_k = 1.0f / K;
    const float seg = b - a;
    const float xs = seg * p.rdn * inv_k;
    const float step = seg * inv_k;
    const float inv_size = e.b.w;
    const float rx = p.rd.x * inv_size, ry = p.rd.y * inv_size, rz = p.rd.z * inv_size;
    float tk[K], ek[K], qx[K], qy[K], qz[K], dsig[K];
    float t = fmaf(0.5f, step, a);
    float trans = 1.f, d = 0.f, X = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        qx[k] = fmaf(t, rx, -e.c.x);
        qy[k] = fmaf(t, ry, -e.c.y);
        qz[k] = fmaf(t, rz, -e.c.z);
        const float v = trilerp(e.g0, e.g1, qx[k], qy[k], qz[k]);
        const float sig = explin(v);
        dsig[k] = v > 1.1f ? 1.f : sig * 0.909090909f;
        const float xk = xs * sig;
        ek[k] = __expf(-xk);
        X += xk;
        tk[k] = t;
        d = fmaf(trans * (1.f - ek[k]), t, d);
        trans *= ek[k];
        t += step;
    }
    if (B2F) {
        // T_known >= 1e-30 here (smaller goes front to back) and T_i <= 1, so
        // trans >= 1e-30 lies in the fast division's 2-ulp range
        T_after = T_known;
        T_i = __fdividef(T_known, trans);
    } else {
        T_i = T_known;
        T_after = T_known * trans;
    }
    const float al = seg_alpha(X, trans);
    w = T_i * al;
    dloc = d;
    float nlen = 0.f;
    nrm = make_float3(0.f, 0.f, 0.f);
    constexpr bool XN = (XM & kXNrm) != 0, XD = (XM & kXDist) != 0, XS = (XM & kXStat) != 0;
    if (XN) nlen = voxel_normal(e.g0, e.g1, nrm);
    if (!B2F) {
        SC0 -= w * e.col.x;
        SC1 -= w * e.col.y;
        SC2 -= w * e.col.z;
        SD -= T_i * d;
        if (XN) {
            SN.x -= w * nrm.x;
            SN.y -= w * nrm.y;
            SN.z -= w * nrm.z;
        }
    }
    dcol[0] = w * g.gC0;
    dcol[1] = w * g.gC1;
    dcol[2] = w * g.gC2;
    // dL/dx_i through C, A and the transmittance of later voxels in D
    float gx = g.gC0 * fmaf(T_after, e.col.x, -SC0) + g.gC1 * fmaf(T_after, e.col.y, -SC1) +
               g.gC2 * fmaf(T_after, e.col.z, -SC2) + g.gA * g.Tfin - g.gD * SD;
    if (XN)
        gx += g.gN0 * fmaf(T_after, nrm.x, -SN.x) + g.gN1 * fmaf(T_after, nrm.y, -SN.y) +
              g.gN2 * fmaf(T_after, nrm.z, -SN.z);
    if (XD) {
        if (g.gL != 0.f) {
            const float m = 0.5f * (a + b);
            const float Wlt = g.Wtot - DS.W - w, Slt = g.Stot - DS.S - w * m;
            cdist = 2.f * (fmaf(m, Wlt, -Slt) + fmaf(-m, DS.W, DS.S)) + 0.666666667f * w * (b - a);
            gx += g.gL * fmaf(T_after, cdist, -DS.R);
        }
    }
    if (XS) prio = fabsf(gx * al / fmaxf(trans, 1e-30f));
    // per-sample depth term, suffix Q_k = sum_{m>k} P_m (1 - e_m) t_m
    float Pk[K + 1];
    Pk[0] = 1.f;
#pragma unroll
    for (int k = 0; k < K; ++k) Pk[k + 1] = Pk[k] * ek[k];
    float Q = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) dgeo[c] = 0.f;
    const float gdT = g.gD * T_i;
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        const float gxk = fmaf(gdT, fmaf(Pk[k + 1], tk[k], -Q), gx);
        const float dv = gxk * xs * dsig[k];
        // trilinear adjoint, the x and y weights folded into dv first
        const float ax1 = dv * qx[k], ax0 = dv - ax1;
        const float b01 = ax0 * qy[k], b00 = ax0 - b01, b11 = ax1 * qy[k], b10 = ax1 - b11;
        const float uz = 1.f - qz[k];
        dgeo[0] = fmaf(b00, uz, dgeo[0]);
        dgeo[1] = fmaf(b00, qz[k], dgeo[1]);
        dgeo[2] = fmaf(b01, uz, dgeo[2]);
        dgeo[3] = fmaf(b01, qz[k], dgeo[3]);
        dgeo[4] = fmaf(b10, uz, dgeo[4]);
        dgeo[5] = fmaf(b10, qz[k], dgeo[5]);
        dgeo[6] = fmaf(b11, uz, dgeo[6]);
        dgeo[7] = fmaf(b11, qz[k], dgeo[7]);
        Q = fmaf(Pk[k] * (1.f - ek[k]), tk[k], Q);
    }
    // normal: dL/dn = w g_N, through the normalisation (I - n n^T) / |grad|
    // and Eq. interp_grad_grad: dgrad/dV_c = (2 x_c - 1, 2 y_c - 1, 2 z_c - 1) / 4
    if (XN && nlen > 0.f) {
        const float dnx = w * g.gN0, dny = w * g.gN1, dnz = w * g.gN2;
        const float dot = dnx * nrm.x + dny * nrm.y + dnz * nrm.z;
        const float il = 0.25f / nlen;
        const float gx_ = (dnx - nrm.x * dot) * il, gy_ = (dny - nrm.y * dot) * il, gz_ = (dnz - nrm.z * dot) * il;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            dgeo[c] += ((c & 4) ? gx_ : -gx_) + ((c & 2) ? gy_ : -gy_) + ((c & 1) ? gz_ : -gz_);
    }
}

// ------------------------------------------------------- gradient records
//
// The gradients of one batch's hits go to per-hit records of kRec floats (8
// corner densities, 3 colour channels) laid out entry by entry: the hits of
// staged entry j get consecutive slots, in pixel order, so a lane writes each
// of its hits' records to a slot of its own with no coordination.  Once the
// hits are done, lane j sums entry j's records and adds the sums to the
// global gradients (one set of atomics per entry and warp).  At most kRecCap
// records are held at a time: a batch with more hits is processed in runs of
// consecutive entries, which keeps every pixel's hits in list order.
constexpr int kRecStride = 12;   // floats per record slot: 11 used, 16-byte aligned
#ifndef SVR_BWD_REC_CAP
#define SVR_BWD_REC_CAP 128
#endif
constexpr int kRecCap = SVR_BWD_REC_CAP;

struct RecSmem {
    float4 rec[kRecCap * kRecStride / 4];
    int off[kBatch];       // first slot of entry j (numbered over the whole batch)
    unsigned pix[kBatch];  // lanes whose pixel hits entry j
};

// Lays out the records of a batch from the lanes' hit masks; lane j returns
// entry j's first slot and end slot, and the batch's record count.
__device__ __forceinline__ int rec_layout(RecSmem &rs, unsigned hits, int &off, int &end) {
    const int lane = threadIdx.x & 31;
    const unsigned pix = warp_transpose(hits);
    int total;
    off = warp_exclusive_scan(__popc(pix), &total);
    end = off + __popc(pix);
    rs.off[lane] = off;
    rs.pix[lane] = pix;
    __syncwarp();
    return total;
}

// Slot, relative to base, of the calling lane's hit on entry k.
__device__ __forceinline__ int rec_slot(const RecSmem &rs, int k, int base) {
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    return rs.off[k] + __popc(rs.pix[k] & lt) - base;
}

// Record: 8 corner-density gradients, 3 colour gradients and the
// subdivision priority term (extras; 0 otherwise).
__device__ __forceinline__ void rec_write(RecSmem &rs, int slot, const float dgeo[8], const float dcol[3],
                                          float prio) {
    float4 *r = rs.rec + slot * (kRecStride / 4);
    r[0] = make_float4(dgeo[0], dgeo[1], dgeo[2], dgeo[3]);
    r[1] = make_float4(dgeo[4], dgeo[5], dgeo[6], dgeo[7]);
    r[2] = make_float4(dcol[0], dcol[1], dcol[2], prio);
}

__device__ __forceinline__ void rec_add(float row[kRecStride], const float4 *r) {
    const float4 a = r[0], b = r[1], c = r[2];
    row[0] += a.x, row[1] += a.y, row[2] += a.z, row[3] += a.w;
    row[4] += b.x, row[5] += b.y, row[6] += b.z, row[7] += b.w;
    row[8] += c.x, row[9] += c.y, row[10] += c.z, row[11] += c.w;
}

// End of the run of entries from k_lo whose records fit in kRecCap slots
// from base (the entries' end slots grow with j, so the run is contiguous).
__device__ __forceinline__ int rec_run_end(int k_lo, int end, int base) {
    const int lane = threadIdx.x & 31;
    const unsigned fit = __ballot_sync(0xffffffffu, lane >= k_lo && end - base <= kRecCap);
    return 32 - __clz(fit);
}

// Adds an entry's summed record to the global gradients of voxel vid; a
// colour channel that the clamp cut (bit clear) has no gradient.
__device__ __forceinline__ void add_row(const float row[kRecStride], int vid, unsigned bits,
                                        const int32_t *__restrict__ corner_idx, float *__restrict__ d_grid,
                                        float *__restrict__ acc_col, float *__restrict__ priority,
                                        DebugBlock *dbg, int64_t n_pts) {
    const int4 *ci = reinterpret_cast<const int4 *>(corner_idx + 8 * (size_t)vid);
    const int4 i0 = __ldg(ci), i1 = __ldg(ci + 1);
    if (!(SVR_IN_BOUNDS(dbg, kDbgGradPoint, i0.x, n_pts) && SVR_IN_BOUNDS(dbg, kDbgGradPoint, i0.y, n_pts) &&
          SVR_IN_BOUNDS(dbg, kDbgGradPoint, i0.z, n_pts) && SVR_IN_BOUNDS(dbg, kDbgGradPoint, i0.w, n_pts) &&
          SVR_IN_BOUNDS(dbg, kDbgGradPoint, i1.x, n_pts) && SVR_IN_BOUNDS(dbg, kDbgGradPoint, i1.y, n_pts) &&
          SVR_IN_BOUNDS(dbg, kDbgGradPoint, i1.z, n_pts) && SVR_IN_BOUNDS(dbg, kDbgGradPoint, i1.w, n_pts)))
        return;
    atomicAdd(d_grid + i0.x, row[0]);
    atomicAdd(d_grid + i0.y, row[1]);
    atomicAdd(d_grid + i0.z, row[2]);
    atomicAdd(d_grid + i0.w, row[3]);
    atomicAdd(d_grid + i1.x, row[4]);
    atomicAdd(d_grid + i1.y, row[5]);
    atomicAdd(d_grid + i1.z, row[6]);
    atomicAdd(d_grid + i1.w, row[7]);
    if (bits & 1u) atomicAdd(acc_col + 3 * (size_t)vid + 0, row[8]);
    if (bits & 2u) atomicAdd(acc_col + 3 * (size_t)vid + 1, row[9]);
    if (bits & 4u) atomicAdd(acc_col + 3 * (size_t)vid + 2, row[10]);
    if (priority) atomicAdd(priority + vid, row[11]);
}

// Lane j in [k_lo, k_hi) sums entry j's records and adds the sums to the
// global gradients of its voxel.
__device__ __forceinline__ void rec_flush(const RecSmem &rs, const Entry *st, int k_lo, int k_hi, int off, int end,
                                          int base, const FrameDev &f, float *__restrict__ d_grid,
                                          float *__restrict__ acc_col, float *__restrict__ priority) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane >= k_lo && lane < k_hi && end > off) {
        float row[kRecStride];
#pragma unroll
        for (int c = 0; c < kRecStride; ++c) row[c] = 0.f;
        for (int r = off - base; r < end - base; ++r) rec_add(row, rs.rec + r * (kRecStride / 4));
        add_row(row, __float_as_int(st[lane].col.w), __float_as_uint(st[lane].pad.x), f.corner_idx, d_grid, acc_col,
                priority, f.debug, f.n_pts);
    }
    __syncwarp();
}

// Mask of staged entries [k_lo, k_hi).
__device__ __forceinline__ unsigned range_mask(int k_lo, int k_hi) {
    const unsigned hi = k_hi >= 32 ? 0xffffffffu : ((1u << k_hi) - 1u);
    return hi & ~((1u << k_lo) - 1u);
}

struct BwdIn {
    const float *d_rgb, *d_depth, *d_alpha, *T;
    const int32_t *last;
    float *d_grid;
    const float *d_normal;  // extras: upstream gradient of the normal image [3][H][W], or NULL
    float *priority;        // extras: [N] subdivision priority, accumulated, or NULL
    const float *d_dist;    // extras: upstream gradient of each ray's distortion loss [H][W], or NULL
    const float *dist;      // extras: the forward's [2][H][W] distortion output (plane 1: sum w m)
    float *max_weight;      // extras: [N] per-voxel maximum of T_i alpha_i (atomicMax), or NULL
};

// Front-to-back gradients for the pixels of an item whose transmittance
// behind their part of the list underflowed (the back-to-front recovery
// T_i = T_(i+1) / (1 - alpha_i) would lose precision): sweep 1 sums the
// part's colour, depth (and normal) from the transmittance in front of it,
// sweep 2 takes the gradients with the sums behind each voxel as total minus
// prefix.
template <int K, int XM>
__device__ __noinline__ void bwd_front_to_back(const FrameDev &f, const ItemList L, int p0, int p1, int idx0,
                                               int last, bool fallback, float T_before, float SC0, float SC1, float SC2,
                                               float SD, NrmSums SN, DistSums DSb, const ViewData vd,
                                               const WarpBlock wb, const PixelRay p, const PixelGrad g, Entry *st,
                                               RecSmem &rs, const BwdIn &in, float *dcol) {
    constexpr bool XN = (XM & kXNrm) != 0, XD = (XM & kXDist) != 0, XS = (XM & kXStat) != 0;
    const int lane = threadIdx.x & 31;
    const int n_fb = lower_pos(L.list, p0, p1, __reduce_max_sync(0xffffffffu, fallback ? last + 1 : idx0));
    // sweep 1: this part's own sums, from the transmittance in front of it
    // (distortion: the part's internal loss and sums of w, w m)
    float T = T_before, Ct0 = 0.f, Ct1 = 0.f, Ct2 = 0.f, Dt = 0.f;
    NrmSums Nt = {0.f, 0.f, 0.f};
    FwdState dp = {};
    for (int base = p0; base < n_fb; base += kBatch) {
        Lookahead cur;
        fetch_vi(cur, L.list, base + lane, base + lane < n_fb);
        fetch_box(cur, vd);
        const unsigned cand = warp_transpose(entry_pixels(cur.valid, cur.vi.x, cur.box, wb));
        stage_ahead(st, vd, cur);
        if (fallback) {
            for (unsigned c = cand; c; c &= c - 1u) {
                const Entry &e = st[__ffs(c) - 1];
                float a, b;
                if (__float_as_int(e.c.w) > last || !slab(e, p, a, b)) continue;
                float trans, dloc, al;
                hit_fwd<K>(e, p, a, b, trans, dloc, al);
                const float w = T * al;
                Ct0 = fmaf(w, e.col.x, Ct0);
                Ct1 = fmaf(w, e.col.y, Ct1);
                Ct2 = fmaf(w, e.col.z, Ct2);
                Dt = fmaf(T, dloc, Dt);
                if (XN) {
                    float3 n;
                    voxel_normal(e.g0, e.g1, n);
                    Nt.x = fmaf(w, n.x, Nt.x);
                    Nt.y = fmaf(w, n.y, Nt.y);
                    Nt.z = fmaf(w, n.z, Nt.z);
                }
                if (XD && g.gL != 0.f) dist_add(dp, w, a, b);
                T *= trans;
            }
        }
        __syncwarp();
    }
    Ct0 += SC0;
    Ct1 += SC1;
    Ct2 += SC2;
    Dt += SD;
    Nt.x += SN.x;
    Nt.y += SN.y;
    Nt.z += SN.z;
    // distortion: sum w dL/dw over this part (its internal pairs twice, its
    // pairs with the voxels in front A and behind C) plus the part's behind
    const float WA = g.Wtot - dp.PW - DSb.W, SA = g.Stot - dp.PS - DSb.S;
    const float Rt = 2.f * dp.LD + 2.f * (dp.PS * WA - dp.PW * SA) + 2.f * (dp.PW * DSb.S - dp.PS * DSb.W) + DSb.R;
    // sweep 2: gradients with the sums behind = total - prefix
    float Tf = T_before, PC0 = 0.f, PC1 = 0.f, PC2 = 0.f, PD = 0.f;
    NrmSums PN = {0.f, 0.f, 0.f};
    float PW = 0.f, PS = 0.f, PR = 0.f;
    for (int base = p0; base < n_fb; base += kBatch) {
        Lookahead cur;
        fetch_vi(cur, L.list, base + lane, base + lane < n_fb);
        fetch_box(cur, vd);
        const unsigned cand = warp_transpose(entry_pixels(cur.valid, cur.vi.x, cur.box, wb));
        stage_ahead(st, vd, cur);
        unsigned hits = 0;
        if (fallback) {
            for (unsigned c = cand; c; c &= c - 1u) {
                const int k = __ffs(c) - 1;
                const Entry &e = st[k];
                float a, b;
                if (__float_as_int(e.c.w) <= last && slab(e, p, a, b)) hits |= 1u << k;
            }
        }
        int off, end;
        const int total = rec_layout(rs, hits, off, end);
        for (int k_lo = 0, rb = 0; rb < total; rb = __shfl_sync(0xffffffffu, off, k_lo)) {
            const int k_hi = rec_run_end(k_lo, end, rb);
            unsigned h = hits & range_mask(k_lo, k_hi);
            while (h != 0) {
                const int k = __ffs(h) - 1;   // staged in increasing list order
                h &= h - 1;
                const Entry &e = st[k];
                float a, b;
                slab(e, p, a, b);
                float T_i, Ta, w, dloc, dgeo[8], dc[3], prio = 0.f, cdist = 0.f;
                float3 n;
                const NrmSums Nb = {Nt.x - PN.x, Nt.y - PN.y, Nt.z - PN.z};
                // the voxel's own w is only known inside hit_grad: pass the
                // sums behind it including its own share and let the
                // distortion term subtract it (see below)
                float w_own = 0.f, m_own = 0.f, c_own = 0.f;
                if (XD && g.gL != 0.f) {
                    float tr, dl, al_;
                    hit_fwd<K>(e, p, a, b, tr, dl, al_);
                    w_own = Tf * al_;
                    m_own = 0.5f * (a + b);
                }
                const DistSums Db = {g.Wtot - WA - PW - w_own, g.Stot - SA - PS - w_own * m_own, 0.f};
                DistSums Dx = Db;
                if (XD && g.gL != 0.f) {
                    // dL/dw of this voxel from the prefix and suffix sums
                    const float Wlt = WA + PW, Slt = SA + PS;
                    c_own = 2.f * (fmaf(m_own, Wlt, -Slt) + fmaf(-m_own, Db.W, Db.S)) +
                            0.666666667f * w_own * (b - a);
                    Dx.R = Rt - PR - w_own * c_own;
                }
                hit_grad<K, false, XM>(e, p, g, a, b, Tf, Ct0 - PC0, Ct1 - PC1, Ct2 - PC2, Dt - PD, Nb, Dx, dgeo,
                                          dc, T_i, Ta, w, dloc, n, prio, cdist);
                PC0 = fmaf(w, e.col.x, PC0);
                PC1 = fmaf(w, e.col.y, PC1);
                PC2 = fmaf(w, e.col.z, PC2);
                PD = fmaf(T_i, dloc, PD);
                if (XS && in.max_weight)
                    atomicMax(reinterpret_cast<int *>(in.max_weight) + __float_as_int(e.col.w), __float_as_int(w));
                if (XN) {
                    PN.x = fmaf(w, n.x, PN.x);
                    PN.y = fmaf(w, n.y, PN.y);
                    PN.z = fmaf(w, n.z, PN.z);
                }
                if (XD && g.gL != 0.f) {
                    PW += w_own;
                    PS = fmaf(w_own, m_own, PS);
                    PR = fmaf(w_own, c_own, PR);
                }
                Tf = Ta;
                rec_write(rs, checked(f.debug, kDbgRecSlot, rec_slot(rs, k, rb), kRecCap), dgeo, dc, prio);
            }
            rec_flush(rs, st, k_lo, k_hi, off, end, rb, f, in.d_grid, dcol, XS ? in.priority : nullptr);
            k_lo = k_hi;
            if (k_lo >= 32) break;
        }
        __syncwarp();
    }
}

template <int K, int XM>
__device__ __forceinline__ void bwd_item(const FrameDev &f, const Item &it, Entry *st, RecSmem &rs,
                                         const BwdIn &in) {
    constexpr bool XN = (XM & kXNrm) != 0, XD = (XM & kXDist) != 0, XS = (XM & kXStat) != 0;
    const ItemView iv = item_view(f, it.g);
    const DevCam &cam = f.views[iv.view];
    const ViewData &vd = iv.vd;
    float *dcol = f.dcol + 3 * (size_t)iv.view * f.n_vox;
    WarpBlock wb;
    const PixelRay p = pixel_ray(cam, iv.tile, it.blk, wb);
    if (wb.smask == 0) return;
    const ItemList L = item_list(f, it.g, it.blk);
    {
        // a block with no entries in this item's part of the list has no hit
        int q0 = 0, q1 = L.n_list;
        if (L.ts.x > 1) seg_range(L, f.blocks_per_tile, it.seg, q0, q1);
        if (q1 <= q0) return;
    }
    const int beg = L.beg;
    const int lane = threadIdx.x & 31;
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t px = (size_t)p.y * cam.W + p.x;
    const size_t o = (size_t)cam.pix_base + px;

    PixelGrad g = {0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int last = beg - 1;
    if (p.inside) {
        if (in.d_rgb) {
            const float *gr = in.d_rgb + 3 * (size_t)cam.pix_base + px;
            g.gC0 = gr[0];
            g.gC1 = gr[HW];
            g.gC2 = gr[2 * HW];
        }
        if (in.d_depth) g.gD = in.d_depth[o];
        if (in.d_alpha) g.gA = in.d_alpha[o];
        if (XN && in.d_normal) {
            const float *gn = in.d_normal + 3 * (size_t)cam.pix_base + px;
            g.gN0 = gn[0];
            g.gN1 = gn[HW];
            g.gN2 = gn[2 * HW];
        }
        g.Tfin = in.T[o];
        if (XD && in.d_dist) {
            g.gL = in.d_dist[o];
            g.Wtot = 1.f - g.Tfin;
            g.Stot = in.dist[2 * (size_t)cam.pix_base + HW + px];
        }
        last = max(beg - 1, min(in.last[o], L.end - 1));   // stay inside the tile's list
    }
    // The part of the list this item covers and the state behind it: the
    // whole list behind which lies T_final bg, or one segment of a split
    // tile with the forward's sums behind it and transmittance around it.
    int p0 = 0, p1 = L.n_list, idx0 = beg;
    float T_after = g.Tfin, T_before = 1.f;
    float SC0 = g.Tfin * f.bg[0], SC1 = g.Tfin * f.bg[1], SC2 = g.Tfin * f.bg[2], SD = 0.f;
    NrmSums SN = {0.f, 0.f, 0.f};
    DistSums DS = {0.f, 0.f, 0.f};
    // every tile takes the hit masks of this sort's forward; a split tile
    // also starts from its segment sums, which must include the normal image
    // and the distortion sums when their gradients are asked for
    {
        const unsigned done = f.status->fwd_done;
        if (done == 0 || (L.ts.x > 1 && ((XN && in.d_normal && !(done & 2u)) || (XD && in.d_dist && !(done & 4u))))) {
            if (lane == 0) atomicOr(&f.status->flags, SVR_FLAG_NO_FORWARD);
            return;
        }
    }
    if (L.ts.x > 1) {
        seg_range(L, f.blocks_per_tile, it.seg, p0, p1);
        idx0 = beg + it.seg * kSegLen;
        const float *q = seg_fields(f, L.ts.y + it.seg, it.blk);
        SC0 = q[0];
        SC1 = q[32];
        SC2 = q[2 * 32];
        SD = q[3 * 32];
        T_after = q[4 * 32];
        T_before = q[5 * 32];
        if (XN) {
            SN.x = q[8 * 32];
            SN.y = q[9 * 32];
            SN.z = q[10 * 32];
        }
        if (XD && in.d_dist) {
            DS.W = q[11 * 32];
            DS.S = q[12 * 32];
            DS.R = q[13 * 32];
        }
    }
    const bool has = p.inside && last >= idx0;
    const bool fallback = has && T_after < 1e-30f;
    const bool active = has && !fallback;
    float *prio_out = XS ? in.priority : nullptr;

    // ---- back to front, over the forward's batches [p0 + 32 k, p0 + 32 k + 32):
    // each pixel's hits in a batch are the forward's hit mask (which tested
    // every candidate of the batch before the pixel stopped) restricted to
    // the entries up to its last voxel
    {
        const int top_all = lower_pos(L.list, p0, p1, __reduce_max_sync(0xffffffffu, active ? last + 1 : idx0));
        const uint32_t *hm = hit_masks(f, L, it);
        int base = p0 + (((top_all - 1 - p0) >> 5) << 5);   // the batch of position top_all - 1
        Lookahead la;
        unsigned m_next = 0u;
        la.valid = false;
        if (top_all > p0) {
            fetch_vi(la, L.list, base + kBatch - 1 - lane, base + kBatch - 1 - lane < top_all);
            m_next = __ldg(hm + base + lane);
        }
        prefetch_record(la, vd);
        for (; top_all > p0 && base >= p0; base -= kBatch) {
            const Lookahead cur = la;
            const unsigned m = m_next;
            if (base - kBatch >= p0) {
                fetch_vi(la, L.list, base - 1 - lane, true);
                m_next = __ldg(hm + base - kBatch + lane);
            } else {
                la.valid = false;
            }
            // staged indices fall with j (lane j: list position base + 31 - j):
            // the first j whose index is <= last
            const int idx_j = cur.valid ? (int)cur.vi.y : INT_MAX;
            int lo = 0, hi = kBatch;
#pragma unroll
            for (int step = 0; step < 6; ++step) {
                const int mid = (lo + hi) >> 1;
                const int v = __shfl_sync(0xffffffffu, idx_j, mid & 31);
                if (lo < hi) {
                    if (v > last) lo = mid + 1;
                    else hi = mid;
                }
            }
            const unsigned hits = active && lo < kBatch ? __brev(m) & (0xffffffffu << lo) : 0u;
            // only the entries some pixel hits are staged (every lane takes
            // part in the reduction)
            const unsigned needed = __reduce_or_sync(0xffffffffu, hits);
            if (cur.valid && ((needed >> lane) & 1u))
                stage_entry(st[lane], (cur.vi.x & 0xE0000000u) | vid_of(vd, cur.vi.x), (int)cur.vi.y, vd.rec);
            __syncwarp();
            prefetch_record(la, vd);
            int off, end;
            const int total = rec_layout(rs, hits, off, end);
            // runs of entries whose records fit; each lane takes its hits in
            // staged order (decreasing list position: back to front)
            for (int k_lo = 0, base = 0; base < total; base = __shfl_sync(0xffffffffu, off, k_lo)) {
                const int k_hi = rec_run_end(k_lo, end, base);
                unsigned h = hits & range_mask(k_lo, k_hi);
                while (h != 0) {
                    const int k = __ffs(h) - 1;
                    h &= h - 1;
                    const Entry &e = st[k];
                    float a, b;
                    slab(e, p, a, b);
                    float T_i, Ta, w, dloc, dgeo[8], dc[3], prio = 0.f, cdist = 0.f;
                    float3 n;
                    hit_grad<K, true, XM>(e, p, g, a, b, T_after, SC0, SC1, SC2, SD, SN, DS, dgeo, dc, T_i, Ta, w,
                                             dloc, n, prio, cdist);
                    SC0 = fmaf(w, e.col.x, SC0);
                    SC1 = fmaf(w, e.col.y, SC1);
                    SC2 = fmaf(w, e.col.z, SC2);
                    SD = fmaf(T_i, dloc, SD);
                    if (XS && in.max_weight)
                        atomicMax(reinterpret_cast<int *>(in.max_weight) + __float_as_int(e.col.w), __float_as_int(w));
                    if (XN) {
                        SN.x = fmaf(w, n.x, SN.x);
                        SN.y = fmaf(w, n.y, SN.y);
                        SN.z = fmaf(w, n.z, SN.z);
                    }
                    if (XD && g.gL != 0.f) {
                        DS.W += w;
                        DS.S = fmaf(w, 0.5f * (a + b), DS.S);
                        DS.R = fmaf(w, cdist, DS.R);
                    }
                    T_after = T_i;
                    rec_write(rs, checked(f.debug, kDbgRecSlot, rec_slot(rs, k, base), kRecCap), dgeo, dc, prio);
                }
                rec_flush(rs, st, k_lo, k_hi, off, end, base, f, in.d_grid, dcol, prio_out);
                k_lo = k_hi;
                if (k_lo >= 32) break;
            }
            __syncwarp();
        }
    }

    // ---- front to back for pixels whose transmittance underflowed (rare:
    // kept out of line so that it does not weigh on the main path's registers)
    if (__any_sync(0xffffffffu, fallback))
        bwd_front_to_back<K, XM>(f, L, p0, p1, idx0, last, fallback, T_before, SC0, SC1, SC2, SD, SN, DS, vd, wb,
                                    p, g, st, rs, in, dcol);
}

template <int K, int XM>
__global__ void __launch_bounds__(kBwdThreads, kBwdMinBlocks) k_render_bwd(FrameDev f, BwdIn in) {
    __shared__ Entry stage[kBwdWarps][kBatch];
    __shared__ RecSmem recs[kBwdWarps];
    const int warp = threadIdx.x >> 5;
    Entry *st = stage[warp];
    const unsigned bpt = (unsigned)f.blocks_per_tile;
    const unsigned n_items = f.status->n_listed * bpt;  // an empty tile has no gradient
    Item it;
    while (next_item(&f.status->bwd_next, n_items, bpt, f.order, it)) {
        bwd_item<K, XM>(f, it, st, recs[warp], in);
        __syncwarp();
    }
}

// Per voxel: dL/dsh[n][c] = sum over views of Y_n(d_v) * dL/dc_{v,c}, over
// the views where the voxel is in view (dL/dc_{v,c} holds only the channels
// that were > 0 before the clamp, Eq. vox_color); zero for a voxel in no view.  Each thread sums its
// voxel's 48 values in registers and stores them to a shared row (rows 52
// floats apart: float4 stores of a quarter warp fall in distinct banks); the
// block then writes its rows as consecutive float4s.
constexpr int kVoxBwdThreads = 128;
constexpr int kShRow = 52;

__global__ void __launch_bounds__(kVoxBwdThreads) k_voxel_bwd(FrameDev f, float *__restrict__ d_sh) {
    __shared__ __align__(16) float rows[kVoxBwdThreads * kShRow];
    const int64_t v0 = (int64_t)blockIdx.x * kVoxBwdThreads;
    const int64_t v = v0 + threadIdx.x;
    if (v < f.n_vox) {
        float o[48];
#pragma unroll
        for (int i = 0; i < 48; ++i) o[i] = 0.f;
        for (int view = 0; view < f.n_views; ++view) {
            const int64_t iv = (int64_t)view * f.n_vox + v;
            if (f.count[iv] == 0) continue;
            const DevCam &cam = f.views[view];
            const float g0 = f.dcol[3 * iv + 0], g1 = f.dcol[3 * iv + 1], g2 = f.dcol[3 * iv + 2];
            float dx = f.centre[3 * v + 0] - cam.ro[0];
            float dy = f.centre[3 * v + 1] - cam.ro[1];
            float dz = f.centre[3 * v + 2] - cam.ro[2];
            const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
            float Y[16];
            sh_basis(dx * inv, dy * inv, dz * inv, Y);
#pragma unroll
            for (int n = 0; n < 16; ++n) {
                o[3 * n + 0] = fmaf(Y[n], g0, o[3 * n + 0]);
                o[3 * n + 1] = fmaf(Y[n], g1, o[3 * n + 1]);
                o[3 * n + 2] = fmaf(Y[n], g2, o[3 * n + 2]);
            }
        }
        float4 *row = reinterpret_cast<float4 *>(rows + threadIdx.x * kShRow);
#pragma unroll
        for (int q = 0; q < 12; ++q) row[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
    __syncthreads();
    const int nv = (int)tmin<int64_t>(kVoxBwdThreads, f.n_vox - v0);
    float4 *out = reinterpret_cast<float4 *>(d_sh + 48 * v0);
    const float4 *src = reinterpret_cast<const float4 *>(rows);
    for (int i = threadIdx.x; i < nv * 12; i += kVoxBwdThreads) {
        const int r = i / 12;
        out[i] = src[r * (kShRow / 4) + (i - 12 * r)];
    }
}

// ---------------------------------------------------------------- launchers

// Persistent grid: as many CTAs as fit on the device at once.
template <class Kern>
static unsigned persistent_grid(Kern kernel, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (sms <= 0) sms = 1;
    if (per_sm <= 0) per_sm = 1;
    return (unsigned)(sms * per_sm);
}

cudaError_t launch_block_lists(const FrameDev &f, int sorted_alt, cudaStream_t s) {
    if (f.total_tiles == 0) return cudaSuccess;
    // at most one CTA per possible entry of the work order, at most as many as
    // are resident at once; they stride over the device-side count
    const int64_t grid = (int64_t)f.total_tiles + f.seg_slots;
    static DeviceCache cache;
    const unsigned resident = device_cached(cache, [] { return persistent_grid(k_block_lists, kListThreads); });
    k_block_lists<<<(unsigned)tmin<int64_t>(grid, resident), kListThreads, 0, s>>>(f, f.vals[sorted_alt]);
    return cudaGetLastError();
}

// Grid size from a lower bound on the work items (every tile has at least
// one segment); the kernels read the exact count from the device.
template <int K, int MODE>
static cudaError_t fwd_k(const FrameDev &f, const FwdOut &out, cudaStream_t s) {
    static DeviceCache cache;
    const unsigned grid = device_cached(cache, [] { return persistent_grid(k_render_fwd<K, MODE>, kThreads); });
    const unsigned items = (unsigned)f.total_tiles * (unsigned)f.blocks_per_tile;
    const unsigned g = tmin<unsigned>(grid, (items + kWarps - 1) / kWarps);
    k_render_fwd<K, MODE><<<g, kThreads, 0, s>>>(f, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || MODE != kModeExtra || !out.max_weight) return e;
    // the later segments of split lists, from their true transmittance
    static DeviceCache cache_w;
    const unsigned grid_w = device_cached(cache_w, [] { return persistent_grid(k_render_maxw<K>, kThreads); });
    e = cudaMemsetAsync(&f.status->maxw_next, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    FwdOut wout = out;
    wout.normal = nullptr;
    wout.dist = nullptr;
    k_render_maxw<K><<<tmin<unsigned>(grid_w, (items + kWarps - 1) / kWarps), kThreads, 0, s>>>(f, wout);
    return cudaGetLastError();
}

template <int K, int XM>
static cudaError_t bwd_k(const FrameDev &f, const BwdIn &in, cudaStream_t s) {
    static DeviceCache cache;
    const unsigned grid =
        device_cached(cache, [] { return persistent_grid(k_render_bwd<K, XM>, kBwdThreads); });
    const unsigned items = (unsigned)f.total_tiles * (unsigned)f.blocks_per_tile;
    const unsigned g = tmin<unsigned>(grid, (items + kBwdWarps - 1) / kBwdWarps);
    k_render_bwd<K, XM><<<g, kBwdThreads, 0, s>>>(f, in);
    return cudaGetLastError();
}

cudaError_t launch_render_fwd(const FrameDev &f, float *rgb, float *depth, float *alpha,
                              float *T_final, int32_t *last, int2 *stats, float *normal, float *max_weight,
                              float *dist, cudaStream_t s) {
    const FwdOut out = {rgb, depth, alpha, T_final, last, stats, normal, max_weight, dist};
    const int mode = stats ? kModeStats : (normal || max_weight) ? kModeExtra : dist ? kModeDist : kModePlain;
    // the work counter is zero here: cleared with the status block, then by
    // the last warp of every launch
    cudaError_t e;
    switch (f.K * 4 + mode) {
        case 4: e = fwd_k<1, kModePlain>(f, out, s); break;
        case 5: e = fwd_k<1, kModeStats>(f, out, s); break;
        case 6: e = fwd_k<1, kModeExtra>(f, out, s); break;
        case 7: e = fwd_k<1, kModeDist>(f, out, s); break;
        case 8: e = fwd_k<2, kModePlain>(f, out, s); break;
        case 9: e = fwd_k<2, kModeStats>(f, out, s); break;
        case 10: e = fwd_k<2, kModeExtra>(f, out, s); break;
        case 11: e = fwd_k<2, kModeDist>(f, out, s); break;
        case 12: e = fwd_k<3, kModePlain>(f, out, s); break;
        case 13: e = fwd_k<3, kModeStats>(f, out, s); break;
        case 14: e = fwd_k<3, kModeExtra>(f, out, s); break;
        case 15: e = fwd_k<3, kModeDist>(f, out, s); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

cudaError_t launch_render_bwd(const FrameDev &f, const float *d_rgb, const float *d_depth,
                              const float *d_alpha, const float *T_final, const int32_t *last, float *d_grid,
                              float *d_sh, const float *d_normal, float *priority, const float *d_dist,
                              const float *dist, float *max_weight, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&f.status->bwd_next, 0, sizeof(unsigned), s);
    if (e == cudaSuccess && f.n_vox > 0)
        e = cudaMemsetAsync(f.dcol, 0, sizeof(float) * 3 * (size_t)f.n_vox * f.n_views, s);
    if (e != cudaSuccess) return e;
    const BwdIn in = {d_rgb, d_depth, d_alpha, T_final, last, d_grid, d_normal, priority, d_dist, dist, max_weight};
    // extras: none; the distortion gradient alone (the training step's); it
    // and the pruning/subdivision statistics (the training step that gathers
    // them); every extra (the normal gradient as well)
    const int xm = d_normal ? 3 : (priority || max_weight) ? 2 : d_dist ? 1 : 0;
    constexpr int kXDS = kXDist | kXStat;
    switch (f.K * 4 + xm) {
        case 4: e = bwd_k<1, 0>(f, in, s); break;
        case 5: e = bwd_k<1, kXDist>(f, in, s); break;
        case 6: e = bwd_k<1, kXDS>(f, in, s); break;
        case 7: e = bwd_k<1, kXAll>(f, in, s); break;
        case 8: e = bwd_k<2, 0>(f, in, s); break;
        case 9: e = bwd_k<2, kXDist>(f, in, s); break;
        case 10: e = bwd_k<2, kXDS>(f, in, s); break;
        case 11: e = bwd_k<2, kXAll>(f, in, s); break;
        case 12: e = bwd_k<3, 0>(f, in, s); break;
        case 13: e = bwd_k<3, kXDist>(f, in, s); break;
        case 14: e = bwd_k<3, kXDS>(f, in, s); break;
        case 15: e = bwd_k<3, kXAll>(f, in, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (f.n_vox > 0) {
        k_voxel_bwd<<<(unsigned)((f.n_vox + kVoxBwdThreads - 1) / kVoxBwdThreads), kVoxBwdThreads, 0, s>>>(f, d_sh);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace svr
