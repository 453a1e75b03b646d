// Stable LSD radix sort of the (key, value) pairs and per-tile ranges.
//
// The pair count lives on the device (written by the count scan); every
// kernel reads it, so the host enqueues the sort without knowing it and the
// sequence can be captured in a CUDA graph.  One pass sorts 8 key bits:
//   k_radix_count     per tile of 4096 pairs: digit histogram -> hist[digit][tile]
//   k_radix_digit     per digit: exclusive scan over the tiles, digit total
//   k_radix_scatter   per tile: stable rank of each pair among the pairs of
//                     its digit (warp match + per-warp counts, in index
//                     order), written to digit base + tile offset + rank
// Pairs with equal keys keep their order (emission order), so sorting the
// value's sign bits first and then the key bits orders pairs by (key, value).
//
//   k_tile_ranges     [begin, end) of each tile id (key >> 48) in the sorted list
#include "svr_internal.cuh"

namespace svr {

// Pairs to sort: the emitted count, or none when the emission was skipped
// because the count exceeded the capacity (the buffers then hold stale data).
__device__ __forceinline__ uint32_t pair_count(const Status *st, int64_t cap) {
    if (st->flags & SVR_FLAG_CAPACITY) return 0u;
    const unsigned long long p = ((unsigned long long)st->n_pairs_hi << 32) | st->n_pairs_lo;
    return (uint32_t)tmin<unsigned long long>(p, (unsigned long long)cap);
}

__device__ __forceinline__ uint32_t digit_of(uint64_t key, uint32_t val, int shift, bool sign_pass) {
    return sign_pass ? (val >> 29) : (uint32_t)((key >> shift) & 0xFFu);
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_count(const uint64_t *__restrict__ keys,
                                                               const uint32_t *__restrict__ vals,
                                                               const Status *st, int64_t cap, int shift,
                                                               bool sign_pass, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    const uint32_t P = pair_count(st, cap);
    const uint32_t nb = (P + kRadixTile - 1) / kRadixTile;
    const int lane = threadIdx.x & 31;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        h[threadIdx.x] = 0;
        // all loads of the tile first, so their latencies overlap
        const uint32_t base = b * kRadixTile;
        uint32_t d[kRadixItems];
#pragma unroll
        for (int r = 0; r < kRadixItems; ++r) {
            const uint32_t i = base + r * kRadixThreads + threadIdx.x;
            d[r] = i < P ? digit_of(keys[i], sign_pass ? vals[i] : 0u, shift, sign_pass) : 256u;
        }
        __syncthreads();
        // one shared atomic per digit value present in the warp
#pragma unroll
        for (int r = 0; r < kRadixItems; ++r) {
            const unsigned peers = __match_any_sync(0xffffffffu, d[r]);
            if (d[r] < 256u && lane == __ffs(peers) - 1) atomicAdd(&h[d[r]], (uint32_t)__popc(peers));
        }
        __syncthreads();
        hist[(size_t)threadIdx.x * nb + b] = h[threadIdx.x];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_radix_digit(uint32_t *__restrict__ hist, const Status *st,
                                                      int64_t cap, uint32_t *__restrict__ digit_tot) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const uint32_t P = pair_count(st, cap);
    const uint32_t nb = (P + kRadixTile - 1) / kRadixTile;
    const int d = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    uint32_t *row = hist + (size_t)d * nb;
    for (uint32_t base = 0; base < nb; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < nb ? row[i] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int w = 0; w < 32; ++w) {
            const uint32_t s = wsum[w];
            wpre += (w < warp) ? s : 0u;
            tot += s;
        }
        if (i < nb) row[i] = carry + wpre + inc - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) digit_tot[d] = carry;
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const Status *st, int64_t cap, int shift, bool sign_pass,
    const uint32_t *__restrict__ hist, const uint32_t *__restrict__ digit_tot) {
    constexpr int kWarps = kRadixThreads / 32;
    __shared__ uint32_t base_d[256];     // global start of each digit in this tile
    __shared__ uint32_t run[256];        // pairs of each digit already placed in this tile
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t wpre[kWarps][256];
    __shared__ uint32_t wsum[kWarps];

    const uint32_t P = pair_count(st, cap);
    const uint32_t nb = (P + kRadixTile - 1) / kRadixTile;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    // exclusive scan of the digit totals (one digit per thread)
    uint32_t tot_d = digit_tot[t];
    uint32_t inc = tot_d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t wp = 0;
    for (int w = 0; w < warp; ++w) wp += wsum[w];
    const uint32_t digit_start = wp + inc - tot_d;

    const unsigned lt_mask = (1u << lane) - 1u;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        base_d[t] = digit_start + hist[(size_t)t * nb + b];
        run[t] = 0;
        for (int w = 0; w < kWarps; ++w) wcnt[w][t] = 0;
        __syncthreads();
        const uint32_t base = b * kRadixTile;
        // all loads of the tile first, so their latencies overlap
        uint64_t keys[kRadixItems];
        uint32_t vals[kRadixItems];
#pragma unroll
        for (int r = 0; r < kRadixItems; ++r) {
            const uint32_t i = base + r * kRadixThreads + t;
            keys[r] = i < P ? kin[i] : 0ull;
            vals[r] = i < P ? vin[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kRadixItems; ++r) {
            const uint32_t i = base + r * kRadixThreads + t;
            const bool valid = i < P;
            const uint64_t key = keys[r];
            const uint32_t val = vals[r];
            const uint32_t d = valid ? digit_of(key, val, shift, sign_pass) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & lt_mask);
            if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
            __syncthreads();
            {
                uint32_t acc = run[t];
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    wpre[w][t] = acc;
                    acc += wcnt[w][t];
                    wcnt[w][t] = 0;
                }
                run[t] = acc;
            }
            __syncthreads();
            if (valid) {
                const uint32_t pos = base_d[d] + wpre[warp][d] + rank;
                kout[pos] = key;
                vout[pos] = val;
            }
        }
        __syncthreads();
    }
}

__global__ void k_tile_ranges(const uint64_t *__restrict__ keys, const Status *st, int64_t cap,
                              uint32_t ntiles, int shift, uint2 *__restrict__ ranges) {
    const uint32_t P = pair_count(st, cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const uint32_t tile = (uint32_t)(keys[i] >> shift);
        if (tile >= ntiles) continue;
        if (i == 0 || (uint32_t)(keys[i - 1] >> shift) != tile) ranges[tile].x = i;
        if (i == P - 1 || (uint32_t)(keys[i + 1] >> shift) != tile) ranges[tile].y = i + 1;
    }
}

// Render work order: one entry (tile, segment) per segment of every tile's
// list.  A list of L > kSegLen entries is split into ceil(L / kSegLen)
// segments of kSegLen consecutive entries, which get consecutive slots for
// their partial sums; a shorter list is one segment without a slot.  Entries
// are grouped by floor(log2(segment length)), longest first, so the heaviest
// work starts early and short segments fill the tail (one CTA; the order
// within a group is arbitrary and results do not depend on it).  Also resets
// the frame's forward-done mark: the segment sums belong to the last sort.
__global__ void __launch_bounds__(1024) k_tile_order(FrameDev f) {
    __shared__ unsigned cnt[33];
    __shared__ unsigned start[33];
    __shared__ unsigned slot_next;
    const int t = threadIdx.x;
    const int ntiles = f.total_tiles;
    if (t < 33) cnt[t] = 0;
    if (t == 0) slot_next = 0;
    __syncthreads();
    for (int i = t; i < ntiles; i += blockDim.x) {
        const uint2 r = f.ranges[i];
        const unsigned len = r.y - r.x;
        unsigned nseg = len > (unsigned)kSegLen ? (len + kSegLen - 1) / kSegLen : 1u;
        unsigned base = 0;
        if (nseg > 1) {
            base = atomicAdd(&slot_next, nseg);
            if ((int64_t)base + nseg > f.seg_slots) nseg = 1, base = 0;  // only past the pair capacity
        }
        const unsigned w = nseg > 1 ? (unsigned)kSegLen : len;
        atomicAdd(&cnt[w ? 32 - __clz(w) : 0], nseg);
        f.tile_seg[i] = make_uint2(nseg, base);
    }
    __syncthreads();
    if (t == 0) {
        unsigned acc = 0;
        for (int b = 32; b >= 0; --b) {
            start[b] = acc;
            acc += cnt[b];
        }
        f.status->n_queue = acc;
        f.status->slots_used = slot_next;
        f.status->fwd_done = 0;
    }
    __syncthreads();
    for (int i = t; i < ntiles; i += blockDim.x) {
        const uint2 r = f.ranges[i];
        const uint2 ts = f.tile_seg[i];
        const unsigned len = r.y - r.x;
        const unsigned w = ts.x > 1 ? (unsigned)kSegLen : len;
        const unsigned pos = atomicAdd(&start[w ? 32 - __clz(w) : 0], ts.x);
        for (unsigned sg = 0; sg < ts.x; ++sg) f.order[pos + sg] = make_uint2((unsigned)i, sg);
    }
}

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t launch_sort(const FrameDev &f, int lo_bit, int hi_bit, bool sign_pass, int *result_alt,
                        cudaStream_t s) {
    *result_alt = 0;
    if (f.capacity == 0) return cudaSuccess;
    const int64_t tiles_cap = (f.capacity + kRadixTile - 1) / kRadixTile;
    const unsigned grid = (unsigned)tmin<int64_t>(tiles_cap, (int64_t)sm_count() * 8);
    int cur = 0;
    auto pass = [&](int shift, bool sp) {
        k_radix_count<<<grid, kRadixThreads, 0, s>>>(f.keys[cur], f.vals[cur], f.status, f.capacity,
                                                    shift, sp, f.hist);
        k_radix_digit<<<256, 1024, 0, s>>>(f.hist, f.status, f.capacity, f.digit_tot);
        k_radix_scatter<<<grid, kRadixThreads, 0, s>>>(f.keys[cur], f.vals[cur], f.keys[cur ^ 1],
                                                      f.vals[cur ^ 1], f.status, f.capacity, shift, sp,
                                                      f.hist, f.digit_tot);
        cur ^= 1;
    };
    if (sign_pass) pass(0, true);
    for (int b = lo_bit; b < hi_bit; b += 8) pass(b, false);
    *result_alt = cur;
    return cudaGetLastError();
}

cudaError_t launch_ranges(const FrameDev &f, int sorted_alt, cudaStream_t s) {
    const int ntiles = f.total_tiles;
    cudaError_t e = cudaMemsetAsync(f.ranges, 0, sizeof(uint2) * (size_t)ntiles, s);
    if (e != cudaSuccess) return e;
    if (f.capacity > 0) {
        const int64_t need = (f.capacity + 255) / 256;
        const unsigned grid = (unsigned)tmin<int64_t>(need, (int64_t)sm_count() * 8);
        k_tile_ranges<<<grid, 256, 0, s>>>(f.keys[sorted_alt], f.status, f.capacity, (uint32_t)ntiles, f.key_shift,
                                           f.ranges);
    }
    k_tile_order<<<1, 1024, 0, s>>>(f);
    return cudaGetLastError();
}

}  // namespace svr
