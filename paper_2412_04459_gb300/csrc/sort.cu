// Tile ranges, render work order and the radix sort of the (key, value)
// pairs by (tile id, Morton order).
//
// The tile id is the most significant digit and is sorted by counting: the
// scan of the per-tile counts gives every tile its range and k_emit writes
// each pair into its tile's range (order within a tile arbitrary).  The
// Morton bits that can differ are then sorted tile by tile:
//   k_tile_order   the tiles' ranges from the scanned counts, and the render
//                  work order: one entry per tile, or per 1024-entry segment
//                  of a longer list, longest first
//   k_sort_small   every list of at most 1024 pairs and every 1024-pair
//                  chunk of a longer list, one at a time per CTA of a
//                  persistent grid: lists of at most 256 pairs by rank, the
//                  others by stable LSD radix passes of 8-bit digits, in
//                  shared memory
//   k_merge_runs   lists longer than 1024 pairs: their sorted chunks merged in
//                  rounds of pairwise stable merges (merge-path partitioning
//                  over the CTA's threads), in shared memory up to 8192 pairs
// The result equals a sort of all pairs by (key, value).
#include "svr_internal.cuh"

namespace svr {

// Render work order: one entry (tile, segment) per segment of every tile's
// list.  A list of L > kSegLen entries is split into ceil(L / kSegLen)
// segments of kSegLen consecutive entries, which get consecutive slots for
// their partial sums; a shorter list is one segment without a slot.  Entries
// are grouped by floor(log2(list length)), longest lists first, so the
// heaviest work starts early and short lists fill the tail (one CTA; the
// order within a group is arbitrary and results do not depend on it).  The
// first segments of the split lists come before all other entries, so the
// long-list merge takes its tiles from the head of the order (status n_long
// of them); the empty tiles' entries come last (status n_listed entries
// precede them), so the kernels with nothing to do for an empty list stop
// there.  Also resets the frame's forward-done mark (the segment sums
// belong to the last sort) and the long-list sort's work counter.
// Group of a list in the work order: floor(log2(length)) + 1, one more for a
// split list, so that every split list (longer than kSegLen) precedes every
// unsplit one; a split list's first segment goes to group kFirstSeg + its
// group, ahead of all others.
constexpr int kOrderGroups = 34;
constexpr int kFirstSeg = kOrderGroups;
__device__ __forceinline__ int order_bucket(unsigned len, unsigned nseg) {
    return len ? 32 - __clz(len) + (nseg > 1 ? 1 : 0) : 0;
}

constexpr int kOrderUnroll = 8;  // tiles per thread whose loads are issued together

__global__ void __launch_bounds__(1024) k_tile_order(FrameDev f) {
    __shared__ unsigned cnt[2 * kOrderGroups];
    __shared__ unsigned start[2 * kOrderGroups];
    __shared__ unsigned slot_next;
    const int t = threadIdx.x, nt = blockDim.x;
    const int ntiles = f.total_tiles;
    const bool over = (f.status->flags & SVR_FLAG_CAPACITY) != 0;
    if (t < 2 * kOrderGroups) cnt[t] = 0;
    if (t == 0) slot_next = 0;
    __syncthreads();
    // ranges: a tile starts at its first sub-bucket; empty tiles, and all
    // tiles when the pairs exceed the capacity, get (0, 0); then each tile's
    // segments and its group's count
    for (int i0 = t; i0 < ntiles; i0 += nt * kOrderUnroll) {
        uint32_t b[kOrderUnroll], e[kOrderUnroll];
#pragma unroll
        for (int u = 0; u < kOrderUnroll; ++u) {
            const int i = i0 + u * nt;
            b[u] = i < ntiles ? f.cursor[i] : 0u;
            e[u] = i < ntiles ? f.tile_end[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kOrderUnroll; ++u) {
            const int i = i0 + u * nt;
            if (i >= ntiles) break;
            const uint2 r = over || e[u] == b[u] ? make_uint2(0u, 0u) : make_uint2(b[u], e[u]);
            f.ranges[i] = r;
            const unsigned len = r.y - r.x;
            unsigned nseg = len > (unsigned)kSegLen ? (len + kSegLen - 1) / kSegLen : 1u;
            unsigned base = 0;
            if (nseg > 1) {
                base = atomicAdd(&slot_next, nseg);
                if ((int64_t)base + nseg > f.seg_slots) nseg = 1, base = 0;  // only past the pair capacity
            }
            const int bk = order_bucket(len, nseg);
            if (nseg > 1) {
                atomicAdd(&cnt[kFirstSeg + bk], 1u);
                atomicAdd(&cnt[bk], nseg - 1);
            } else {
                atomicAdd(&cnt[bk], 1u);
            }
            f.tile_seg[i] = make_uint2(nseg, base);
        }
    }
    __syncthreads();
    if (t == 0) {
        unsigned acc = 0;
        for (int b = 2 * kOrderGroups - 1; b >= 0; --b) {
            start[b] = acc;
            acc += cnt[b];
            if (b == kFirstSeg) f.status->n_long = acc;
        }
        f.status->n_queue = acc;
        f.status->n_listed = acc - cnt[0];  // group 0 (the empty lists) is last
        f.status->slots_used = slot_next;
        f.status->fwd_done = 0;
        f.status->sort_next = 0;
    }
    __syncthreads();
    // each thread reads back its own tiles' ranges and segments
    for (int i0 = t; i0 < ntiles; i0 += nt * kOrderUnroll) {
        uint2 r[kOrderUnroll], ts[kOrderUnroll];
#pragma unroll
        for (int u = 0; u < kOrderUnroll; ++u) {
            const int i = i0 + u * nt;
            r[u] = i < ntiles ? f.ranges[i] : make_uint2(0u, 0u);
            ts[u] = i < ntiles ? f.tile_seg[i] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kOrderUnroll; ++u) {
            const int i = i0 + u * nt;
            if (i >= ntiles) break;
            const int bk = order_bucket(r[u].y - r[u].x, ts[u].x);
            if (ts[u].x > 1) {
                f.order[atomicAdd(&start[kFirstSeg + bk], 1u)] = make_uint2((unsigned)i, 0u);
                const unsigned pos = atomicAdd(&start[bk], ts[u].x - 1) - 1;
                for (unsigned sg = 1; sg < ts[u].x; ++sg) f.order[pos + sg] = make_uint2((unsigned)i, sg);
            } else {
                f.order[atomicAdd(&start[bk], 1u)] = make_uint2((unsigned)i, 0u);
            }
        }
    }
}

// -------------------------------------------------------- per-tile radix

constexpr int kSmallThreads = 256;
constexpr int kSmallPairs = kSegLen;    // lists up to this length: one CTA each, shared memory
constexpr int kIdxBits = 16;            // low bits of a sort word: index (or value rank) in the list

// Digit counts and per-warp offsets of one counting pass.
template <int THREADS>
struct RadixTables {
    uint32_t run[256];                  // next output position of each digit
    uint32_t wcnt[THREADS / 32][256];   // pairs of each digit in each warp's part of a round
    uint32_t wpre[THREADS / 32][256];   // output position of each warp's first pair of each digit
    uint32_t wsum[8];
};

template <int THREADS>
__device__ void radix_tables_clear(RadixTables<THREADS> &tb) {
    for (int i = threadIdx.x; i < (THREADS / 32) * 256; i += THREADS) (&tb.wcnt[0][0])[i] = 0;
}

// One stable counting pass of n <= 4 * THREADS words src -> dst by the 8-bit
// digit at bit `shift` (warp-private multisplit).  Warp w ranks its own
// contiguous 128 words in four rounds of 32 with warp-local digit counters
// (warp match: a word's rank is the count of its digit in the warp's earlier
// words), so the ranking needs no CTA barrier; one scan over the (digit,
// warp) counts in digit-major order then gives every (digit, warp) its first
// output position, and each word goes there plus its rank.  Words of lower
// warps and earlier rounds precede, so equal digits keep their order.
template <int THREADS, class Src, class Dst>
__device__ void radix_pass(Src src, Dst dst, int n, int shift, RadixTables<THREADS> &tb) {
    constexpr int W = THREADS / 32;
    static_assert(THREADS == 256, "one counter column per digit and thread");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t *cnt = tb.wcnt[warp];
#pragma unroll
    for (int k = 0; k < 256 / 32; ++k) cnt[lane + 32 * k] = 0;
    __syncwarp();
    uint64_t word[4];
    uint32_t dig[4], rank[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = 128 * warp + 32 * r + lane;
        const bool valid = i < n;
        word[r] = valid ? src(i) : 0ull;
        const uint32_t d = valid ? (uint32_t)(word[r] >> shift) & 0xFFu : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t prior = valid ? cnt[d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[d] = prior + __popc(peers);
        __syncwarp();
        dig[r] = d;
        rank[r] = prior + __popc(peers & lt);
    }
    __syncthreads();
    // thread t = digit t: its total over the warps, exclusive scan over the
    // digits, then each warp's first position for the digit
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) tot += tb.wcnt[w][t];
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tb.wsum[warp] = inc;
    __syncthreads();
    uint32_t pos = inc - tot;
#pragma unroll
    for (int w = 0; w < W; ++w) pos += w < warp ? tb.wsum[w] : 0u;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t c = tb.wcnt[w][t];
        tb.wpre[w][t] = pos;
        pos += c;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = 128 * warp + 32 * r + lane;
        if (i < n) dst(tb.wpre[warp][dig[r]] + rank[r], word[r], i);
    }
    __syncthreads();
}

// Sorts one tile's n <= cap pairs (gk, gv) in shared memory: each pair
// becomes the word (Morton bits << kIdxBits | its index), stable LSD passes
// over the Morton bits [lo_bit, lo_bit + nbits) sort the words, and the
// pairs are gathered by index from ok/ov (their unsorted copy).  Within a
// tile the Morton bits differ between any two pairs below max level 16;
// with max level 16 (ties) the low word bits hold the pair's value rank
// instead, from a first sort of (value << kIdxBits | index), so that equal
// keys end in value order.
template <int THREADS>
__device__ void tile_radix_sort(uint64_t *__restrict__ gk, uint32_t *__restrict__ gv, int n, int lo_bit, int nbits,
                                bool ties, uint64_t *w0, uint64_t *w1, const uint64_t *ok, const uint32_t *ov,
                                uint16_t *inv, RadixTables<THREADS> &tb) {
    const uint64_t mask = nbits >= 64 ? ~0ull : (1ull << nbits) - 1ull;
    auto from0 = [&](int i) { return w0[i]; };
    auto from1 = [&](int i) { return w1[i]; };
    auto to0 = [&](uint32_t p, uint64_t w, int) { w0[p] = w; };
    auto to1 = [&](uint32_t p, uint64_t w, int) { w1[p] = w; };
    radix_tables_clear<THREADS>(tb);
    int cur = 0;  // words in w0
    if (ties) {
        for (int i = threadIdx.x; i < n; i += THREADS) w0[i] = ((uint64_t)ov[i] << kIdxBits) | (uint64_t)i;
        for (int b = 0; b < 32; b += 8, cur ^= 1) {
            if (cur == 0) radix_pass<THREADS>(from0, to1, n, kIdxBits + b, tb);
            else radix_pass<THREADS>(from1, to0, n, kIdxBits + b, tb);
        }
        const uint64_t *ws = cur ? w1 : w0;
        uint64_t *wd = cur ? w0 : w1;
        for (int p = threadIdx.x; p < n; p += THREADS) inv[p] = (uint16_t)(ws[p] & 0xFFFFu);
        __syncthreads();
        for (int p = threadIdx.x; p < n; p += THREADS) {
            const int i = inv[p];
            wd[i] = (((ok[i] >> lo_bit) & mask) << kIdxBits) | (uint64_t)p;  // p = value rank of pair i
        }
        cur ^= 1;
    } else {
        for (int i = threadIdx.x; i < n; i += THREADS)
            w0[i] = (((ok[i] >> lo_bit) & mask) << kIdxBits) | (uint64_t)i;
    }
    __syncthreads();
    for (int b = 0; b < nbits; b += 8, cur ^= 1) {
        if (cur == 0) radix_pass<THREADS>(from0, to1, n, kIdxBits + b, tb);
        else radix_pass<THREADS>(from1, to0, n, kIdxBits + b, tb);
    }
    const uint64_t *ws = cur ? w1 : w0;
    for (int p = threadIdx.x; p < n; p += THREADS) {
        const int low = (int)(ws[p] & 0xFFFFu);
        const int i = ties ? inv[low] : low;
        gk[p] = ok[i];
        gv[p] = ov[i];
    }
}

// Sorts one tile's n <= kSmallThreads pairs (gk, gv) by rank: thread t
// holds pair t and its sort word (Morton bits << kIdxBits | t, as the radix
// passes build it), and its output position is the number of words below its
// own.  The words are distinct (each holds its index), so this is the order
// the stable radix passes give, without their fixed cost per pass; most tile
// lists are this short.  Not for max level 16, whose words need the value.
__device__ __forceinline__ void rank_sort(uint64_t *__restrict__ gk, uint32_t *__restrict__ gv, int n, int lo_bit,
                                          uint64_t mask, uint64_t *w) {
    const int t = threadIdx.x;
    uint64_t k = 0ull, wt = 0ull;
    uint32_t v = 0u;
    if (t < n) {
        k = gk[t];
        v = gv[t];
        wt = (((k >> lo_bit) & mask) << kIdxBits) | (uint64_t)t;
        w[t] = wt;
    }
    __syncthreads();
    if (t < n) {
        int r = 0;
#pragma unroll 8
        for (int j = 0; j < n; ++j) r += w[j] < wt ? 1 : 0;
        gk[r] = k;
        gv[r] = v;
    }
}

constexpr int kRankPairs = kSmallThreads;  // lists up to this length: sorted by rank

// Every list of at most kSmallPairs pairs, and every kSegLen-pair chunk of a
// longer list (merged afterwards): a persistent grid of CTAs takes the
// work-order entries in turn (the count is the device's, so no CTA is
// launched for the entries the capacity allows but the frame does not have).
__global__ void __launch_bounds__(kSmallThreads) k_sort_small(FrameDev f, int lo_bit, int nbits, bool ties) {
    __shared__ uint64_t w[2][kSmallPairs];
    __shared__ uint64_t ok[kSmallPairs];
    __shared__ uint32_t ov[kSmallPairs];
    __shared__ RadixTables<kSmallThreads> tb;
    __shared__ uint16_t inv[kSmallPairs];
    const unsigned nq = f.status->n_listed, G = gridDim.x;  // empty lists need no sort
    const uint64_t mask = nbits >= 64 ? ~0ull : (1ull << nbits) - 1ull;
    // the next entry's range and the one after's order record are fetched
    // one item ahead, so that only the first item waits for them
    const uint2 zero = make_uint2(0u, 0u);
    uint2 q_next = blockIdx.x < nq ? f.order[blockIdx.x] : zero;
    uint2 rg_next = blockIdx.x < nq ? f.ranges[q_next.x] : zero;
    uint2 q_after = blockIdx.x + G < nq ? f.order[blockIdx.x + G] : zero;
    for (unsigned e = blockIdx.x; e < nq; e += G) {
        const uint2 q = q_next, rg = rg_next;
        q_next = q_after;
        rg_next = e + G < nq ? f.ranges[q_next.x] : zero;
        q_after = e + 2 * G < nq ? f.order[e + 2 * G] : zero;
        if (!SVR_IN_BOUNDS(f.debug, kDbgRange, rg.y, f.capacity + 1)) continue;
        const int L = (int)(rg.y - rg.x);
        int c0, n;
        if (L <= kSmallPairs) {
            c0 = (int)rg.x;
            n = L;
        } else if (f.tile_seg[q.x].x > 1) {
            c0 = (int)rg.x + (int)q.y * kSegLen;
            n = min(kSegLen, (int)rg.y - c0);
        } else {
            continue;
        }
        if (n < 2) continue;
        uint64_t *gk = f.keys[0] + c0;
        uint32_t *gv = f.vals[0] + c0;
        if (!ties && n <= kRankPairs) {
            rank_sort(gk, gv, n, lo_bit, mask, w[0]);
        } else {
            for (int i = threadIdx.x; i < n; i += kSmallThreads) ok[i] = gk[i], ov[i] = gv[i];
            __syncthreads();
            tile_radix_sort<kSmallThreads>(gk, gv, n, lo_bit, nbits, ties, w[0], w[1], ok, ov, inv, tb);
        }
        __syncthreads();  // shared memory is reused by the next entry
    }
}

__device__ __forceinline__ bool pair_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
    return ka < kb || (ka == kb && va < vb);
}

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
// key/value buffer.  CTAs take the split tiles from a counter: the first
// n_long work-order entries are their first segments, longest lists first.
__global__ void __launch_bounds__(kMergeThreads) k_merge_runs(FrameDev f) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ unsigned entry;
    const unsigned n_long = f.status->n_long;
    for (;;) {
        if (threadIdx.x == 0) entry = atomicAdd(&f.status->sort_next, 1u);
        __syncthreads();
        const unsigned e = entry;
        __syncthreads();
        if (e >= n_long) return;
        const uint2 q = f.order[e];  // a split tile's first segment
        const uint2 rg = f.ranges[q.x];
        if (!SVR_IN_BOUNDS(f.debug, kDbgRange, rg.y, f.capacity + 1)) continue;
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

static unsigned sm_count() {
    static DeviceCache cache;
    return device_cached(cache, [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return (unsigned)(n > 0 ? n : 1);
    });
}

cudaError_t launch_order(const FrameDev &f, cudaStream_t s) {
    k_tile_order<<<1, 1024, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_tile_sort(const FrameDev &f, int lo_bit, int nbits, bool ties, cudaStream_t s) {
    if (f.capacity == 0) return cudaSuccess;
    // at most one CTA per possible work-order entry, at most as many as are
    // resident at once; they stride over the device-side count
    const unsigned grid = (unsigned)((int64_t)f.total_tiles + f.seg_slots);
    static DeviceCache small_cache;
    const unsigned resident = device_cached(small_cache, [] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_small, kSmallThreads, 0);
        return sm_count() * (unsigned)(per_sm > 0 ? per_sm : 1);
    });
    k_sort_small<<<tmin(grid, resident), kSmallThreads, 0, s>>>(f, lo_bit, nbits, ties);
    // the shared-memory opt-in is a per-device function attribute
    static DeviceCache attr_set;
    cudaError_t e = cudaSuccess;
    device_cached(attr_set, [&e] {
        e = cudaFuncSetAttribute(k_merge_runs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMergeSmemBytes);
        return e == cudaSuccess ? 1u : 0u;
    });
    if (e != cudaSuccess) return e;
    k_merge_runs<<<tmin(grid, sm_count()), kMergeThreads, kMergeSmemBytes, s>>>(f);
    return cudaGetLastError();
}

}  // namespace svr
