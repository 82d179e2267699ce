// Step-kernel instantiations: BF16 deviation storage, FP32 collision.
#include "sc_step_inst.cuh"
cudaError_t scgb::launch_step_bf16(const StepLaunch &l, const StepArgs<float> &a) {
  return launch_any<__nv_bfloat16, float>(l, a);
}
const void *scgb::batched_kernel_bf16(int lattice, int stencil, int tile_y, bool t1, size_t *smem) {
  return batched_any<__nv_bfloat16, float>(lattice, stencil, tile_y, t1, smem);
}
const void *scgb::batched_staged_kernel_bf16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                               size_t *smem) {
  return batched_staged_any<__nv_bfloat16, float>(tile_y, stages, blocks_per_sm, self_on, t1, smem);
}
cudaError_t scgb::staged_occupancy_bf16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                       int *blocks) {
  return staged_occupancy<__nv_bfloat16, float>(tile_y, stages, blocks_per_sm, self_on, t1, blocks);
}
cudaError_t scgb::generic_occupancy_bf16(int lattice, int stencil, int tile_y, bool t1, int *blocks) {
  return generic_occupancy<__nv_bfloat16, float>(lattice, stencil, tile_y, t1, blocks);
}
const void *scgb::persistent_staged_kernel_bf16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                              size_t *smem) {
  return persistent_staged_any<__nv_bfloat16, float>(tile_y, stages, blocks_per_sm, self_on, t1, smem);
}
