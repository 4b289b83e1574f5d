// Counting sort of the grain store by zone key: exclusive scan of the key
// counts, scatter of (id, source) pairs, an id sort inside every key and a
// gather of the store columns (keys are computed by the geometry-specific
// sort_keys kernel).  The sorted order is deterministic: by key, then id.
#include "dust_internal.h"

namespace dust {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

int64_t scan_block_sums_size(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

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

// Phase 1: sum of each tile.
__global__ void scan_reduce_kernel(const int32_t *data, int64_t n, int32_t *block_sums)
{
    __shared__ int32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += data[base + k];
    int32_t total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Phase 2: exclusive scan of the tile sums in one block.
__global__ void scan_sums_kernel(int32_t *block_sums, int64_t nb)
{
    __shared__ int32_t ws[32];
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

// Phase 3: exclusive scan inside each tile plus the tile offset.
__global__ void scan_apply_kernel(int32_t *data, int64_t n, const int32_t *block_sums)
{
    __shared__ int32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? data[base + k] : 0;
        s += v[k];
    }
    int32_t total;
    int32_t run = block_exclusive_scan(s, ws, total) + block_sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) data[base + k] = run;
        run += v[k];
    }
}

cudaError_t launch_exclusive_scan(int32_t *data, int64_t n, int32_t *block_sums, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, block_sums);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(block_sums, nb);
    scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, block_sums);
    return cudaGetLastError();
}

// Scatter of (id, source position) pairs to their key segments.  Positions
// inside a segment come from atomics (arbitrary order); the segment sort
// below puts every segment in grain-id order, so the sorted store is
// reproducible.
template <typename Real>
__global__ void sort_scatter_pairs_kernel(const SortArgs<Real> A)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gi < A.src.n;
    const int32_t key = valid ? A.key[gi] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&A.cursor[key], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!valid) return;
    const int32_t pos = base + __popc(peers & ((1u << lane) - 1u));
    A.pair_id[pos] = A.src.id[gi];
    A.pair_src[pos] = (int32_t)gi;
}

// One thread per key: insertion sort of the key's (id, source) pairs by id.
template <typename Real>
__global__ void sort_segments_kernel(const SortArgs<Real> A)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.nkeys1) return;
    const int32_t b = A.count[k], e = A.count[k + 1];
    for (int32_t u = b + 1; u < e; ++u) {
        const int32_t id = A.pair_id[u], src = A.pair_src[u];
        int32_t j = u - 1;
        while (j >= b) {
            const int32_t idj = A.pair_id[j];
            if (idj <= id) break;
            A.pair_id[j + 1] = idj;
            A.pair_src[j + 1] = A.pair_src[j];
            --j;
        }
        A.pair_id[j + 1] = id;
        A.pair_src[j + 1] = src;
    }
}

// Gather every store column into sorted order (coalesced writes; the
// sources are nearly in order because grains move little between sorts).
template <typename Real>
__global__ void sort_gather_kernel(const SortArgs<Real> A)
{
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= A.src.n) return;
    const int32_t src = A.pair_src[pos];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        A.dst.q[d][pos] = A.src.q[d][src];
        A.dst.p[d][pos] = A.src.p[d][src];
    }
    A.dst.id[pos] = A.pair_id[pos];
    if (A.src.species) A.dst.species[pos] = A.src.species[src];
    if (A.src.param) A.dst.param[pos] = A.src.param[src];
}

template <typename Real>
cudaError_t launch_sort_scatter(const SortArgs<Real> &a, cudaStream_t s, bool gather)
{
    if (a.src.n == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((a.src.n + 255) / 256);
    sort_scatter_pairs_kernel<Real><<<nb, 256, 0, s>>>(a);
    sort_segments_kernel<Real><<<(unsigned)((a.nkeys1 + 255) / 256), 256, 0, s>>>(a);
    if (gather) sort_gather_kernel<Real><<<nb, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_sort_scatter<float>(const SortArgs<float> &, cudaStream_t, bool);
template cudaError_t launch_sort_scatter<double>(const SortArgs<double> &, cudaStream_t, bool);

}  // namespace dust
