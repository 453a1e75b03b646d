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
//                  chunk of a longer list: bitonic sort in shared memory
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

// Sorts the n pairs at (gk, gv) by (key, value) in shared memory (sk, sv hold
// N = pow2_at_least(n) pairs; the padding sorts last): bitonic network, one
// compare-exchange per thread and step.
template <int THREADS>
__device__ void smem_sort(uint64_t *__restrict__ gk, uint32_t *__restrict__ gv, int n, uint64_t *sk, uint32_t *sv) {
    const int N = pow2_at_least(n);
    for (int i = threadIdx.x; i < N; i += THREADS) {
        sk[i] = i < n ? gk[i] : ~0ull;
        sv[i] = i < n ? gv[i] : ~0u;
    }
    __syncthreads();
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < N / 2; t += THREADS) {
                const int i = 2 * t - (t & (stride - 1));  // the pair (i, i + stride) of step stride
                const int l = i + stride;
                const uint64_t ki = sk[i], kl = sk[l];
                const uint32_t vi = sv[i], vl = sv[l];
                const bool up = (i & size) == 0;
                if (pair_less(kl, vl, ki, vi) == up) {
                    sk[i] = kl, sk[l] = ki;
                    sv[i] = vl, sv[l] = vi;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += THREADS) {
        gk[i] = sk[i];
        gv[i] = sv[i];
    }
}

// A whole list of at most kSmallPairs pairs, or one kSegLen-pair chunk of a
// longer list (merged afterwards); one CTA per work-order entry.
__global__ void __launch_bounds__(kSmallThreads) k_sort_small(FrameDev f) {
    __shared__ uint64_t sk[kSmallPairs];
    __shared__ uint32_t sv[kSmallPairs];
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
    smem_sort<kSmallThreads>(f.keys[0] + c0, f.vals[0] + c0, n, sk, sv);
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

cudaError_t launch_tile_sort(const FrameDev &f, cudaStream_t s) {
    if (f.capacity == 0) return cudaSuccess;
    // one CTA per possible work-order entry; those past the device-side count exit
    const unsigned grid = (unsigned)((int64_t)f.total_tiles + f.seg_slots);
    k_sort_small<<<grid, kSmallThreads, 0, s>>>(f);
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
