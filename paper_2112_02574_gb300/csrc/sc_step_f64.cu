// Step-kernel instantiations: FP64 deviation storage, FP64 collision (the
// instantiation the parity tests compare with the FP64 oracle most tightly).
#include "sc_step_inst.cuh"
cudaError_t scgb::launch_step_f64(const StepLaunch &l, const StepArgs<double> &a) { return launch_any<double, double>(l, a); }
const void *scgb::batched_kernel_f64(int lattice, int stencil, int tile_y, bool t1, size_t *smem) {
  return batched_any<double, double>(lattice, stencil, tile_y, t1, smem);
}
const void *scgb::batched_staged_kernel_f64(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                               size_t *smem) {
  return batched_staged_any<double, double>(tile_y, stages, blocks_per_sm, self_on, t1, smem);
}
cudaError_t scgb::staged_occupancy_f64(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                       int *blocks) {
  return staged_occupancy<double, double>(tile_y, stages, blocks_per_sm, self_on, t1, blocks);
}
cudaError_t scgb::generic_occupancy_f64(int lattice, int stencil, int tile_y, bool t1, int *blocks) {
  return generic_occupancy<double, double>(lattice, stencil, tile_y, t1, blocks);
}
const void *scgb::persistent_staged_kernel_f64(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                              size_t *smem) {
  return persistent_staged_any<double, double>(tile_y, stages, blocks_per_sm, self_on, t1, smem);
}
