// The step kernels of the two geometries a batch can run as one persistent
// launch (x-z shearing boxes in the orbital-advection frame, x-y Cartesian
// boxes) and the persistent kernels themselves.  Both inline the same tile
// function; this unit is compiled without the contraction of separate
// multiplies and adds into fused multiply-adds (-fmad=false, see build.py),
// so that the two kernels round every operation alike and a batch gives the
// results of its instances stepped one at a time, bit for bit.  The fused
// multiply-adds the tile function asks for explicitly (the packed gather and
// deposit sums) stay.
#include "dust_batch.cuh"

namespace dust {

template cudaError_t launch_step_slab<GEOM_SB, 1, 1>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_step_slab<GEOM_CART, 2, 1>(const TiledArgs<float> &, cudaStream_t);

template int batch_persistent_grid<GEOM_SB, 1, 1>(size_t);
template cudaError_t launch_batch_persistent<GEOM_SB, 1, 1>(const BatchDev &, size_t, int, cudaStream_t);
template int batch_persistent_grid<GEOM_SB, 1, 1, 32, 1, 16>(size_t);
template cudaError_t launch_batch_persistent<GEOM_SB, 1, 1, 32, 1, 16>(const BatchDev &, size_t, int, cudaStream_t);
template int batch_persistent_grid<GEOM_SB, 1, 1, 16, 1, 16>(size_t);
template cudaError_t launch_batch_persistent<GEOM_SB, 1, 1, 16, 1, 16>(const BatchDev &, size_t, int, cudaStream_t);
template int batch_persistent_grid<GEOM_CART, 2, 1>(size_t);
template cudaError_t launch_batch_persistent<GEOM_CART, 2, 1>(const BatchDev &, size_t, int, cudaStream_t);

}  // namespace dust
