// Tile ranges, render work order and the per-tile sort of the (key, value)
// pairs.
//
// Pairs arrive grouped by tile (k_emit writes each tile's pairs into its own
// range, in no particular order), so each tile's range is sorted on its own,
// in shared memory, by (key, value) (the keys of one tile share the tile id):
//   k_tile_order   the tiles' ranges from the scanned counts, and the render
//                  work order: one entry per tile, or per 1024-entry segment
//                  of a longer list, longest first
//   k_sort_small   one CTA per list of at most 1024 pairs, and per 1024-pair
//                  chunk of a longer list: bitonic sort, warp shuffles for
//                  the short strides, shared memory for the long ones
//   k_merge_runs   lists longer than 1024 pairs: their sorted chunks merged
//                  in rounds of pairwise merges (merge-path partitioning over
//                  the CTA's threads), in shared memory up to 8192 pairs
// The result equals a sort of all pairs by (key, value).
#include "svr_internal.cuh"

namespace svr {

// Render work order: one entry (tile, segment) per segment of every tile's
// list.  A list of L > kSegLen entries is split into ceil(L / kSegLen)
// segments of kSegLen consecutive entries, which get consecutive slots for
// their partial sums; a shorter list is one segment without a slot.  Entries
// are grouped by floor(log2(list length)), longest lists first, so the
// heaviest work starts early and short lists fill the tail (one CTA; the
// order within a group is arbitrary and results do not depend on it).  Also
// resets the frame's forward-done mark (the segment sums belong to the last
// sort) and the merge's work counter.
// Group of a list in the work order: floor(log2(length)) + 1, one more for a
// split list, so that every split list (longer than kSegLen) precedes every
// unsplit one.
__device__ __forceinline__ int order_bucket(unsigned len, unsigned nseg) {
    return len ? 32 - __clz(len) + (nseg > 1 ? 1 : 0) : 0;
}

__global__ void __launch_bounds__(1024) k_tile_order(FrameDev f) {
    __shared__ unsigned cnt[34];
    __shared__ unsigned start[34];
    __shared__ unsigned slot_next;
    const int t = threadIdx.x;
    const int ntiles = f.total_tiles;
    // ranges: a tile starts at its first sub-bucket; empty tiles, and all
    // tiles when the pairs exceed the capacity, get (0, 0)
    const bool over = (f.status->flags & SVR_FLAG_CAPACITY) != 0;
    for (int i = t; i < ntiles; i += blockDim.x) {
        const uint32_t b = f.cursor[i], e = f.tile_end[i];
        f.ranges[i] = over || e == b ? make_uint2(0u, 0u) : make_uint2(b, e);
    }
    if (t < 34) cnt[t] = 0;
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
        atomicAdd(&cnt[order_bucket(len, nseg)], nseg);
        f.tile_seg[i] = make_uint2(nseg, base);
    }
    __syncthreads();
    if (t == 0) {
        unsigned acc = 0;
        for (int b = 33; b >= 0; --b) {
            start[b] = acc;
            acc += cnt[b];
        }
        f.status->n_queue = acc;
        f.status->slots_used = slot_next;
        f.status->fwd_done = 0;
        f.status->merge_next = 0;
    }
    __syncthreads();
    for (int i = t; i < ntiles; i += blockDim.x) {
        const uint2 r = f.ranges[i];
        const uint2 ts = f.tile_seg[i];
        const unsigned len = r.y - r.x;
        const unsigned pos = atomicAdd(&start[order_bucket(len, ts.x)], ts.x);
        for (unsigned sg = 0; sg < ts.x; ++sg) f.order[pos + sg] = make_uint2((unsigned)i, sg);
    }
}

// ------------------------------------------------------------ bitonic sort

constexpr int kSmallThreads = 512;
constexpr int kSmallPairs = kSegLen;

__device__ __forceinline__ bool pair_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
    return ka < kb || (ka == kb && va < vb);
}

__device__ __forceinline__ int pow2_at_least(int n) {
    return n <= 1 ? 1 : 1 << (32 - __clz(n - 1));
}

// Compare-exchange of a warp-held element with the element `stride` lanes
// away (stride < 32): the element at index i keeps the smaller of the two
// when (i & stride) == 0 matches the direction `up`, else the larger.
__device__ __forceinline__ void cx_shfl(uint64_t &x, int i, int stride, bool up) {
    const uint64_t p = __shfl_xor_sync(0xffffffffu, x, stride);
    const bool keep_min = ((i & stride) == 0) == up;
    if ((p < x) == keep_min) x = p;
}

// Bitonic sort of N (power of two, 64 <= N <= kSmallPairs) distinct 64-bit
// words.  Warp w holds elements 64w + lane (a) and 64w + 32 + lane (b) in
// registers: steps of stride < 32 are warp shuffles, stride 32 an exchange
// within the lane, and only strides >= 64 go through shared memory (sx).
__device__ void bitonic_words(uint64_t &a, uint64_t &b, int N, uint64_t *sx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool active = warp < N / 64;  // warps past the padded length only join the barriers
    const int ia = 64 * warp + lane, ib = ia + 32;
    for (int size = 2; size <= N; size <<= 1) {
        if (size > 64) {
            if (active) sx[ia] = a, sx[ib] = b;
            __syncthreads();
            for (int stride = size >> 1; stride >= 64; stride >>= 1) {
                for (int t = threadIdx.x; t < N / 2; t += kSmallThreads) {
                    const int i = 2 * t - (t & (stride - 1));
                    const int l = i + stride;
                    const uint64_t xi = sx[i], xl = sx[l];
                    if ((xl < xi) == ((i & size) == 0)) sx[i] = xl, sx[l] = xi;
                }
                __syncthreads();
            }
            if (active) a = sx[ia], b = sx[ib];
            __syncthreads();
        }
        if (active) {
            const bool up_a = (ia & size) == 0, up_b = (ib & size) == 0;
            int stride = size >> 1;
            if (stride >= 32) {  // a and b are each other's partner (ia has bit 32 clear)
                if ((b < a) == up_a) {
                    const uint64_t t = a;
                    a = b, b = t;
                }
                stride = 16;
            }
            for (; stride > 0; stride >>= 1) {
                cx_shfl(a, ia, stride, up_a);
                cx_shfl(b, ib, stride, up_b);
            }
        }
    }
}

// Sorts the n <= kSmallPairs pairs at (gk, gv) of one tile by (key, value).
// The keys of a tile share the tile id, so the order is that of bits
// [lo_bit, lo_bit + nbits) of the key.  Below max level 16 these bits differ
// between any two pairs of a tile, and each pair is sorted as the word
// (bits << 10 | its index), then gathered by index.  With max level 16
// (ties: equal bits possible) the word is (bits << 16 | rank of the value
// among the tile's values), the ranks coming from a first sort of
// (value << 10 | index).
__device__ void chunk_sort(uint64_t *__restrict__ gk, uint32_t *__restrict__ gv, int n, int lo_bit, int nbits,
                           bool ties, uint64_t *sx, uint64_t *ok, uint32_t *ov, uint16_t *inv) {
    const int N = max(64, pow2_at_least(n));
    const int warp = threadIdx.x >> 5;
    const bool active = warp < N / 64;
    const int ia = 64 * warp + (threadIdx.x & 31), ib = ia + 32;
    const uint64_t mask = nbits >= 64 ? ~0ull : (1ull << nbits) - 1ull;
    for (int i = threadIdx.x; i < n; i += kSmallThreads) ok[i] = gk[i], ov[i] = gv[i];
    __syncthreads();
    uint64_t a = ~0ull, b = ~0ull;
    if (ties) {
        if (ia < n) a = ((uint64_t)ov[ia] << 10) | (uint64_t)ia;
        if (ib < n) b = ((uint64_t)ov[ib] << 10) | (uint64_t)ib;
        bitonic_words(a, b, N, sx);
        __syncthreads();
        uint32_t *rank = reinterpret_cast<uint32_t *>(sx);  // sx is free until the next sort
        if (active) {
            if (ia < n) rank[a & 1023u] = (uint32_t)ia, inv[ia] = (uint16_t)(a & 1023u);
            if (ib < n) rank[b & 1023u] = (uint32_t)ib, inv[ib] = (uint16_t)(b & 1023u);
        }
        __syncthreads();
        a = ia < n ? (((ok[ia] >> lo_bit) & mask) << 16) | rank[ia] : ~0ull;
        b = ib < n ? (((ok[ib] >> lo_bit) & mask) << 16) | rank[ib] : ~0ull;
        __syncthreads();
    } else {
        if (ia < n) a = (((ok[ia] >> lo_bit) & mask) << 10) | (uint64_t)ia;
        if (ib < n) b = (((ok[ib] >> lo_bit) & mask) << 10) | (uint64_t)ib;
    }
    bitonic_words(a, b, N, sx);
    __syncthreads();
    if (active) sx[ia] = a, sx[ib] = b;  // position p: the word of the pair that sorts p-th
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
        const uint64_t w = sx[i];
        const int src = ties ? (int)inv[w & 0xFFFFu] : (int)(w & 1023u);
        gk[i] = ok[src];
        gv[i] = ov[src];
    }
}

// A whole list of at most kSmallPairs pairs, or one kSegLen-pair chunk of a
// longer list (merged afterwards); one CTA per work-order entry.
__global__ void __launch_bounds__(kSmallThreads) k_sort_small(FrameDev f, int lo_bit, int nbits, bool ties) {
    __shared__ uint64_t sx[kSmallPairs];
    __shared__ uint64_t ok[kSmallPairs];
    __shared__ uint32_t ov[kSmallPairs];
    __shared__ uint16_t inv[kSmallPairs];
    if (blockIdx.x >= f.status->n_queue) return;
    const uint2 q = f.order[blockIdx.x];
    const uint2 rg = f.ranges[q.x];
    const int L = (int)(rg.y - rg.x);
    int c0, n;
    if (L <= kSmallPairs) {
        c0 = (int)rg.x;
        n = L;
    } else if (f.tile_seg[q.x].x > 1) {
        c0 = (int)rg.x + (int)q.y * kSegLen;
        n = min(kSegLen, (int)rg.y - c0);
    } else {
        return;
    }
    if (n < 2) return;
    chunk_sort(f.keys[0] + c0, f.vals[0] + c0, n, lo_bit, nbits, ties, sx, ok, ov, inv);
}

// ----------------------------------------------------------- merge of runs

constexpr int kMergeThreads = 1024;
constexpr int kMergePairs = 8192;  // longest list merged in shared memory (2 x 96 KB)
constexpr size_t kMergeSmemBytes = (size_t)kMergePairs * 2 * (sizeof(uint64_t) + sizeof(uint32_t));

// One round: the runs of width w of (sk, sv)[0, L) merged pairwise into
// (dk, dv); thread t writes a contiguous share of the outputs, finding its
// start in each pair of runs by a merge-path binary search (ties: first run).
__device__ void merge_round(const uint64_t *sk, const uint32_t *sv, uint64_t *dk, uint32_t *dv, int L, int w) {
    const int per = (L + kMergeThreads - 1) / kMergeThreads;
    int o = threadIdx.x * per;
    const int o_end = min(L, o + per);
    while (o < o_end) {
        const int p0 = o / (2 * w) * (2 * w);
        const int mid = min(L, p0 + w), pend = min(L, p0 + 2 * w);
        const int stop = min(o_end, pend);
        const int k = o - p0, lenA = mid - p0, lenB = pend - mid;
        int lo = max(0, k - lenB), hi = min(k, lenA);
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            // A[m] goes before B[k - 1 - m] unless B's is strictly smaller
            if (pair_less(sk[mid + k - 1 - m], sv[mid + k - 1 - m], sk[p0 + m], sv[p0 + m])) hi = m;
            else lo = m + 1;
        }
        int ia = p0 + lo, ib = mid + (k - lo);
        for (; o < stop; ++o) {
            const bool take_a = ib >= pend || (ia < mid && !pair_less(sk[ib], sv[ib], sk[ia], sv[ia]));
            if (take_a) {
                dk[o] = sk[ia];
                dv[o] = sv[ia++];
            } else {
                dk[o] = sk[ib];
                dv[o] = sv[ib++];
            }
        }
    }
}

// Lists longer than kSmallPairs: their sorted kSegLen-pair chunks merged in
// place, in shared memory up to kMergePairs pairs, else through the second
// key/value buffer.  CTAs take work-order entries from a counter; the split
// lists come first in that order, longest first.
__global__ void __launch_bounds__(kMergeThreads) k_merge_runs(FrameDev f) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ unsigned entry;
    const unsigned nq = f.status->n_queue;
    for (;;) {
        if (threadIdx.x == 0) entry = atomicAdd(&f.status->merge_next, 1u);
        __syncthreads();
        const unsigned e = entry;
        __syncthreads();
        if (e >= nq) return;
        const uint2 q = f.order[e];
        const uint2 ts = f.tile_seg[q.x];
        if (ts.x < 2) return;  // unsplit lists follow all split ones: nothing left to merge
        if (q.y != 0) continue;
        const uint2 rg = f.ranges[q.x];
        const int L = (int)(rg.y - rg.x);
        uint64_t *gk = f.keys[0] + rg.x;
        uint32_t *gv = f.vals[0] + rg.x;
        const bool in_smem = L <= kMergePairs;
        uint64_t *k[2];
        uint32_t *v[2];
        if (in_smem) {
            k[0] = reinterpret_cast<uint64_t *>(dyn);
            k[1] = k[0] + kMergePairs;
            v[0] = reinterpret_cast<uint32_t *>(k[1] + kMergePairs);
            v[1] = v[0] + kMergePairs;
            for (int i = threadIdx.x; i < L; i += kMergeThreads) {
                k[0][i] = gk[i];
                v[0][i] = gv[i];
            }
            __syncthreads();
        } else {
            k[0] = gk, k[1] = f.keys[1] + rg.x, v[0] = gv, v[1] = f.vals[1] + rg.x;
        }
        int cur = 0;
        for (int w = kSegLen; w < L; w *= 2, cur ^= 1) {
            merge_round(k[cur], v[cur], k[cur ^ 1], v[cur ^ 1], L, w);
            __syncthreads();
        }
        if (in_smem || cur == 1) {
            for (int i = threadIdx.x; i < L; i += kMergeThreads) {
                gk[i] = k[cur][i];
                gv[i] = v[cur][i];
            }
        }
        __syncthreads();
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

cudaError_t launch_order(const FrameDev &f, cudaStream_t s) {
    k_tile_order<<<1, 1024, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_tile_sort(const FrameDev &f, int lo_bit, int nbits, bool ties, cudaStream_t s) {
    if (f.capacity == 0) return cudaSuccess;
    // one CTA per possible work-order entry; those past the device-side count exit
    const unsigned grid = (unsigned)((int64_t)f.total_tiles + f.seg_slots);
    k_sort_small<<<grid, kSmallThreads, 0, s>>>(f, lo_bit, nbits, ties);
    // the shared-memory opt-in is a per-device function attribute
    static unsigned long long attr_set = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !((attr_set >> dev) & 1ull)) {
        cudaError_t e = cudaFuncSetAttribute(k_merge_runs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kMergeSmemBytes);
        if (e != cudaSuccess) return e;
        if (dev < 64) attr_set |= 1ull << dev;
    }
    k_merge_runs<<<tmin(grid, (unsigned)sm_count()), kMergeThreads, kMergeSmemBytes, s>>>(f);
    return cudaGetLastError();
}

}  // namespace svr
