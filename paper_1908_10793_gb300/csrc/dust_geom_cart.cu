// Instantiations of the step and sort kernels for one geometry.
#include "dust_slab.cuh"

namespace dust {

template cudaError_t launch_step_per_grain<float, GEOM_CART, 0>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_step_per_grain<float, GEOM_CART, 1>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_step_per_grain<double, GEOM_CART, 0>(const StepArgs<double> &, cudaStream_t);
template cudaError_t launch_step_per_grain<double, GEOM_CART, 1>(const StepArgs<double> &, cudaStream_t);
template cudaError_t launch_step_tiled<float, GEOM_CART, 0>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_step_tiled<float, GEOM_CART, 1>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_step_tiled<double, GEOM_CART, 0>(const TiledArgs<double> &, cudaStream_t);
template cudaError_t launch_step_tiled<double, GEOM_CART, 1>(const TiledArgs<double> &, cudaStream_t);
template cudaError_t launch_step_slab<GEOM_CART, 0, 0>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_step_slab<GEOM_CART, 0, 1>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_step_slab<GEOM_CART, 2, 0>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_predict_slab<GEOM_CART, 0>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_predict_slab<GEOM_CART, 2>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_zone_keys<GEOM_CART>(const SortArgs<float> &, cudaStream_t);
template cudaError_t launch_sort_keys<float, GEOM_CART>(const SortArgs<float> &, cudaStream_t);
template cudaError_t launch_sort_keys<double, GEOM_CART>(const SortArgs<double> &, cudaStream_t);
template cudaError_t launch_predict_tiled<float, GEOM_CART, 0>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_predict_tiled<float, GEOM_CART, 1>(const TiledArgs<float> &, cudaStream_t);
template cudaError_t launch_predict_tiled<double, GEOM_CART, 0>(const TiledArgs<double> &, cudaStream_t);
template cudaError_t launch_predict_tiled<double, GEOM_CART, 1>(const TiledArgs<double> &, cudaStream_t);
template cudaError_t launch_predict_gas<float, GEOM_CART, 0>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_predict_gas<float, GEOM_CART, 1>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_predict_gas<double, GEOM_CART, 0>(const StepArgs<double> &, cudaStream_t);
template cudaError_t launch_predict_gas<double, GEOM_CART, 1>(const StepArgs<double> &, cudaStream_t);

template cudaError_t launch_deposit_mass<GEOM_CART>(const GridDev &, const SpeciesDev &, int, int64_t,
                                                   const double *const[3], const uint8_t *,
                                                   unsigned long long *, unsigned int *, cudaStream_t);

}  // namespace dust
