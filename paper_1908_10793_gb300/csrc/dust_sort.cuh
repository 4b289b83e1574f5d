// Device functions of the zone sort (counting sort by zone key, then id):
// the scan of the key counts, the scatter of (id, source) pairs, the id sort
// inside each key and the block sort of long segments.  Each takes a
// virtual block index, so that the per-context kernels (dust_sort.cu) and
// the batched persistent kernel (dust_batch.cu) run the same code.
#pragma once

#include "dust_internal.h"

namespace dust {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;



__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *warp_sums, int32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;  // inclusive
    }
    __syncthreads();
    total = warp_sums[(blockDim.x >> 5) - 1];
    const int32_t before = warp > 0 ? warp_sums[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

// The scan in three phases over chunks of blockDim.x * kScanItems counts
// (device functions of a virtual block index, so that the batched
// persistent kernel runs the same code).
// Phase 1: sum of chunk vb.
__device__ __forceinline__ void scan_reduce_block(const int32_t *data, int64_t n, int32_t *block_sums,
                                                  int64_t vb, int32_t *ws)
{
    const int64_t base = (vb * blockDim.x + threadIdx.x) * kScanItems;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += data[base + k];
    int32_t total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) block_sums[vb] = total;
}

// Phase 2: exclusive scan of the nb chunk sums by one block.
__device__ __forceinline__ void scan_sums_block(int32_t *block_sums, int64_t nb, int32_t *ws)
{
    int32_t carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int32_t v = i < nb ? block_sums[i] : 0;
        int32_t total;
        const int32_t ex = block_exclusive_scan(v, ws, total);
        if (i < nb) block_sums[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
}

// Phase 3: exclusive scan inside chunk vb plus the chunk's offset; copy, if
// given, receives the same offsets (the scatter's cursors).
__device__ __forceinline__ void scan_apply_block(int32_t *data, int64_t n, const int32_t *block_sums,
                                                 int64_t vb, int32_t *ws, int32_t *copy)
{
    const int64_t base = (vb * blockDim.x + threadIdx.x) * kScanItems;
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? data[base + k] : 0;
        s += v[k];
    }
    int32_t total;
    int32_t run = block_exclusive_scan(s, ws, total) + block_sums[vb];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) {
            data[base + k] = run;
            if (copy) copy[base + k] = run;
        }
        run += v[k];
    }
}

// Scatter of (id, source position) pairs to their key segments.  Positions
// inside a segment come from atomics (arbitrary order); the segment sort
// below puts every segment in grain-id order, so the sorted store is
// reproducible.  A warp takes kScatterItems x 32 consecutive grains and
// issues all their loads, then all their cursor atomics, before it uses a
// result, so that the round trips overlap.
constexpr int kScatterItems = 4;

template <class SA>
__device__ __forceinline__ void scatter_pairs_block(const SA &A, int64_t vb)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (vb * blockDim.x + (threadIdx.x - lane)) * kScatterItems;
    if (w0 >= A.src.n) return;  // whole warp past the end
    int32_t key[kScatterItems], id[kScatterItems], base[kScatterItems], first[kScatterItems];
#pragma unroll
    for (int r = 0; r < kScatterItems; ++r) {
        const int64_t gi = w0 + 32 * r + lane;
        key[r] = gi < A.src.n ? A.key[gi] : -1;  // keys are >= 0
        id[r] = gi < A.src.n ? A.src.id[gi] : 0;
    }
    // runs of equal keys on consecutive lanes (keys arrive nearly sorted):
    // one cursor atomic per run, positions inside the run by lane.  The
    // lanes past the end form one run of key -1 that takes no atomic.
#pragma unroll
    for (int r = 0; r < kScatterItems; ++r) {
        const int32_t prev = __shfl_up_sync(FULL, key[r], 1);
        const bool start = lane == 0 || prev != key[r];
        const unsigned starts = __ballot_sync(FULL, start);
        first[r] = 31 - __clz(starts & ((2u << lane) - 1u));  // this lane's run start
        const unsigned later = starts & ~((2u << lane) - 1u);
        const int end = later ? __ffs(later) - 1 : 32;
        base[r] = 0;
        if (start && key[r] >= 0) base[r] = atomicAdd(&A.cursor[key[r]], end - lane);
    }
#pragma unroll
    for (int r = 0; r < kScatterItems; ++r) {
        const int32_t b = __shfl_sync(FULL, base[r], first[r]);
        if (key[r] >= 0) {
            const int32_t pos = b + (lane - first[r]);
            A.pair_id[pos] = id[r];
            A.pair_src[pos] = (int32_t)(w0 + 32 * r + lane);
        }
    }
}

// Sort by id of the (id, source) pairs of every key.  A warp takes 32
// consecutive keys; their segments are contiguous, so the warp stages them
// in shared memory with coalesced loads, places each pair by its rank in its
// key's segment there, and writes them back.  When the warp's
// segments hold more than kSegStage pairs in total, segments of at most
// kSmallSeg pairs are insertion-sorted in place in global memory (bounded
// cost) and longer ones are listed for the block sort below.
constexpr int kSegThreads = 256;
constexpr int kSegStage = 512;  // pairs staged per warp
constexpr int kSmallSeg = 32;

__device__ __forceinline__ void insertion_sort_pairs(int32_t *id, int32_t *src, int32_t b, int32_t e)
{
    for (int32_t u = b + 1; u < e; ++u) {
        const int32_t x = id[u], y = src[u];
        int32_t j = u - 1;
        while (j >= b) {
            const int32_t idj = id[j];
            if (idj <= x) break;
            id[j + 1] = idj;
            src[j + 1] = src[j];
            --j;
        }
        id[j + 1] = x;
        src[j + 1] = y;
    }
}

// sid / ssrc: kSegStage pairs per warp of the block, in shared memory
template <class SA>
__device__ __forceinline__ void segments_block(const SA &A, int64_t vb, int32_t (*sid)[kSegStage],
                                               int32_t (*ssrc)[kSegStage])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = vb * blockDim.x + threadIdx.x;
    const int64_t k0 = k - lane;
    // keys 0 .. nsort - 1 are zones; key nsort (removed grains) is left as
    // the scatter placed it
    const int64_t nsort = A.nkeys1 - 1;
    if (k0 >= nsort) return;  // whole warp past the zone keys
    const int64_t klast = min(k0 + 32, nsort);  // one past the warp's last key
    const int32_t W0 = A.count[k0], W1 = A.count[klast];
    const bool mine = k < nsort;
    const int32_t b = mine ? A.count[k] : W1, e = mine ? A.count[k + 1] : W1;
    if (W1 - W0 > kSegStage) {
        if (mine && e - b <= kSmallSeg) insertion_sort_pairs(A.pair_id, A.pair_src, b, e);
        else if (mine) A.big[1 + atomicAdd(&A.big[0], 1)] = (int32_t)k;
        return;
    }
    const unsigned FULL = 0xffffffffu;
    // all loads of a half first, then its shared stores: the loads' round
    // trips overlap
    constexpr int kHalf = kSegStage / 64;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int32_t rid[kHalf], rsrc[kHalf];
#pragma unroll
        for (int r = 0; r < kHalf; ++r) {
            const int32_t u = W0 + lane + 32 * (r + h * kHalf);
            if (u < W1) {
                rid[r] = A.pair_id[u];
                rsrc[r] = A.pair_src[u];
            }
        }
#pragma unroll
        for (int r = 0; r < kHalf; ++r) {
            const int32_t u = W0 + lane + 32 * (r + h * kHalf);
            if (u < W1) {
                sid[warp][u - W0] = rid[r];
                ssrc[warp][u - W0] = rsrc[r];
            }
        }
    }
    __syncwarp(FULL);
    // each staged pair goes straight to its place in its key's segment: the
    // segment is found by a binary search over the lanes' segment starts
    // (nondecreasing; lanes past the zone keys hold the end), and the place
    // is the segment start plus the number of smaller ids in the segment (ids
    // are unique); the loads of the count are independent, unlike an
    // insertion sort's
    const int32_t n = W1 - W0;
    const int32_t st = (mine ? b : W1) - W0, en = (mine ? e : W1) - W0;
    for (int32_t r0 = 0; r0 < n; r0 += 32) {
        const int32_t u = r0 + lane;
        int lo = 0, hi = 32;  // the last lane whose segment starts at or before u
#pragma unroll
        for (int it = 0; it < 5; ++it) {
            const int mid = (lo + hi) >> 1;
            if (__shfl_sync(FULL, st, mid) <= u) lo = mid;
            else hi = mid;
        }
        const int32_t sb = __shfl_sync(FULL, st, lo), se = __shfl_sync(FULL, en, lo);
        if (u < n) {
            const int32_t x = sid[warp][u];
            int32_t rank = 0;
            for (int32_t v = sb; v < se; ++v) rank += sid[warp][v] < x ? 1 : 0;
            A.pair_id[W0 + sb + rank] = x;
            A.pair_src[W0 + sb + rank] = ssrc[warp][u];
        }
    }
}

// Block sort by id of the long zone segments the segment sort listed (a
// dense clump puts thousands of grains in one zone).  One block per segment:
// chunks of kBigChunk pairs are sorted in shared memory by a bitonic
// network, then merge passes double the sorted runs, ping-ponging between
// the pair arrays and the scratch.  Ids are unique, so an element's place in
// the merged run is its index in its own run plus the number of smaller ids
// in the other run (a binary search).  Work O(L log L) per segment of L.
constexpr int kBigThreads = 1024;
constexpr int kBigChunk = 4096;
constexpr int kBigSortBlocks = 152;  // one per SM of a GB300

__device__ __forceinline__ int32_t count_less(const int32_t *v, int32_t len, int32_t x)
{
    int32_t lo = 0, hi = len;  // first index with v[index] >= x
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (v[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Items vb, vb + vgrid, ... of the list; sid / ssrc: kBigChunk pairs in
// shared memory.
template <class SA>
__device__ __forceinline__ void big_segments_block(const SA &A, int32_t vb, int32_t vgrid, int32_t *sid,
                                                   int32_t *ssrc)
{
    const int32_t nbig = A.big[0];
    for (int32_t item = vb; item < nbig; item += vgrid) {
        const int32_t key = A.big[1 + item];
        const int32_t b = A.count[key], L = A.count[key + 1] - b;
        // 1. sorted chunks
        for (int32_t c0 = 0; c0 < L; c0 += kBigChunk) {
            const int32_t m = min(kBigChunk, L - c0);
            int32_t P = 2;
            while (P < m) P <<= 1;
            for (int32_t i = threadIdx.x; i < P; i += blockDim.x) {
                sid[i] = i < m ? A.pair_id[b + c0 + i] : 0x7fffffff;  // pads sort last
                ssrc[i] = i < m ? A.pair_src[b + c0 + i] : 0;
            }
            __syncthreads();
            for (int32_t k = 2; k <= P; k <<= 1) {
                for (int32_t j = k >> 1; j > 0; j >>= 1) {
                    for (int32_t i = threadIdx.x; i < P; i += blockDim.x) {
                        const int32_t l = i ^ j;
                        if (l > i) {
                            const int32_t x = sid[i], y = sid[l];
                            if ((x > y) == ((i & k) == 0)) {
                                sid[i] = y;
                                sid[l] = x;
                                const int32_t t = ssrc[i];
                                ssrc[i] = ssrc[l];
                                ssrc[l] = t;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
                A.pair_id[b + c0 + i] = sid[i];
                A.pair_src[b + c0 + i] = ssrc[i];
            }
            __syncthreads();
        }
        // 2. merge passes
        int32_t *fid = A.pair_id + b, *fsrc = A.pair_src + b;
        int32_t *tid = A.tmp_id + b, *tsrc = A.tmp_src + b;
        for (int32_t w = kBigChunk; w < L; w <<= 1) {
            for (int32_t u = threadIdx.x; u < L; u += blockDim.x) {
                const int32_t run = u / w;
                const int32_t p0 = (run & ~1) * w;
                const int32_t a1 = min(p0 + w, L), b1 = min(p0 + 2 * w, L);
                const int32_t x = fid[u];
                const int32_t pos = (run & 1) ? p0 + (u - a1) + count_less(fid + p0, a1 - p0, x)
                                              : u + count_less(fid + a1, b1 - a1, x);
                tid[pos] = x;
                tsrc[pos] = fsrc[u];
            }
            __syncthreads();
            int32_t *t0 = fid, *t1 = fsrc;
            fid = tid; fsrc = tsrc;
            tid = t0; tsrc = t1;
        }
        if (fid != A.pair_id + b) {
            for (int32_t u = threadIdx.x; u < L; u += blockDim.x) {
                A.pair_id[b + u] = fid[u];
                A.pair_src[b + u] = fsrc[u];
            }
        }
        __syncthreads();
    }
}

}  // namespace dust
