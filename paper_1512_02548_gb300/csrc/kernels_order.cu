// One GLL order of the σ-Laplace path: compiled once per order with -DSEM_ORDER=P by the build,
// so that the order-templated kernels build in parallel.  Instantiates the host entry points
// declared in sem_internal.cuh for that order.
#include "laplace_device.cuh"

#ifndef SEM_ORDER
#error "compile with -DSEM_ORDER=<GLL order>"
#endif

namespace semgb {
template cudaError_t upload_tables_impl<SEM_ORDER>(const double*, const double*);
template cudaError_t launch_geometry_impl<SEM_ORDER>(const DevGeom&, const double*, bool, cudaStream_t);
template cudaError_t launch_apply_elem_impl<SEM_ORDER>(const DevGeom&, const double*, double*, double*, cudaStream_t);
template cudaError_t pcg_occupancy_impl<SEM_ORDER>(int, size_t, int*);
template cudaError_t launch_pcg_impl<SEM_ORDER>(int, const DevGeom&, const PcgArgs&, int, size_t, cudaStream_t);
template cudaError_t launch_prec_setup_impl<SEM_ORDER>(const DevGeom&, const PrecSetup&, cudaStream_t);
template cudaError_t launch_apply_tile_impl<SEM_ORDER>(int, const DevGeom&, const void*, void*, cudaStream_t);
template cudaError_t stage_occupancy_impl<SEM_ORDER>(int, int, size_t, int*);
template cudaError_t launch_stage_impl<SEM_ORDER>(int, int, const StageArgs&, int, size_t, cudaStream_t);
template cudaError_t cluster_fit_impl<SEM_ORDER>(int, int, int, size_t, int*);
template cudaError_t launch_stage_cluster_impl<SEM_ORDER>(int, int, const StageArgs&, int, int, size_t, cudaStream_t);
}  // namespace semgb
