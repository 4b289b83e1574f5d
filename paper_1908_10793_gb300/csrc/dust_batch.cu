// Shared-memory sizes of the batched persistent kernel (dust_batch.cuh).
#include "dust_batch.cuh"

namespace dust {

size_t batch_tile_smem(const GridDev &g) { return slab_smem_bytes(g); }

size_t batch_sort_smem()
{
    // segment sort: kSegStage (id, source) pairs per warp; block sort:
    // kBigChunk pairs
    return std::max((size_t)2 * (kSegThreads / 32) * kSegStage, (size_t)2 * kBigChunk) * sizeof(int32_t);
}

}  // namespace dust
