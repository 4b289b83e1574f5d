// Counting sort of the grain store by zone key: exclusive scan of the key
// counts, scatter of (id, source) pairs, an id sort inside every key and a
// gather of the store columns (keys are computed by the geometry-specific
// sort_keys kernel).  The live grains' order is deterministic: by key, then
// id.  Removed grains (the last key) come after them in the scatter's order:
// nothing is computed from them, and sorting that segment, which grows with
// every removal, would make the sort's cost grow with the run's length.
#include "dust_sort.cuh"

namespace dust {

// chunk sums for chunks of at least 256 threads x kScanItems counts
int64_t scan_block_sums_size(int64_t n) { return (n + 256 * kScanItems - 1) / (256 * kScanItems) + 1; }

__global__ void scan_reduce_kernel(const int32_t *data, int64_t n, int32_t *block_sums)
{
    __shared__ int32_t ws[32];
    scan_reduce_block(data, n, block_sums, blockIdx.x, ws);
}

__global__ void scan_sums_kernel(int32_t *block_sums, int64_t nb)
{
    __shared__ int32_t ws[32];
    scan_sums_block(block_sums, nb, ws);
}

__global__ void scan_apply_kernel(int32_t *data, int64_t n, const int32_t *block_sums)
{
    __shared__ int32_t ws[32];
    scan_apply_block(data, n, block_sums, blockIdx.x, ws, nullptr);
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

template <typename Real>
__global__ void sort_scatter_pairs_kernel(const SortArgs<Real> A)
{
    scatter_pairs_block(A, blockIdx.x);
}

template <typename Real>
__global__ void __launch_bounds__(kSegThreads) sort_segments_kernel(const SortArgs<Real> A)
{
    __shared__ int32_t sid[kSegThreads / 32][kSegStage];
    __shared__ int32_t ssrc[kSegThreads / 32][kSegStage];
    segments_block(A, blockIdx.x, sid, ssrc);
}

template <typename Real>
__global__ void __launch_bounds__(kBigThreads) sort_big_segments_kernel(const SortArgs<Real> A)
{
    __shared__ int32_t sid[kBigChunk];
    __shared__ int32_t ssrc[kBigChunk];
    big_segments_block(A, blockIdx.x, gridDim.x, sid, ssrc);
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
    const unsigned nbs = (unsigned)((a.src.n + 256 * kScatterItems - 1) / (256 * kScatterItems));
    sort_scatter_pairs_kernel<Real><<<nbs, 256, 0, s>>>(a);
    sort_segments_kernel<Real><<<(unsigned)((a.nkeys1 + kSegThreads - 1) / kSegThreads), kSegThreads, 0, s>>>(a);
    // long segments, if any (the kernel reads their count on the device)
    sort_big_segments_kernel<Real><<<kBigSortBlocks, kBigThreads, 0, s>>>(a);
    if (gather) sort_gather_kernel<Real><<<nb, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_sort_scatter<float>(const SortArgs<float> &, cudaStream_t, bool);
template cudaError_t launch_sort_scatter<double>(const SortArgs<double> &, cudaStream_t, bool);

}  // namespace dust
