// Step-kernel instantiations: FP32 deviation storage, FP32 collision.
#include "sc_step_inst.cuh"
cudaError_t scgb::launch_step_f32(const StepLaunch &l, const StepArgs<float> &a) { return launch_any<float, float>(l, a); }
const void *scgb::batched_kernel_f32(int lattice, int stencil, int tile_y, bool t1, size_t *smem) {
  return batched_any<float, float>(lattice, stencil, tile_y, t1, smem);
}
const void *scgb::batched_staged_kernel_f32(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                               size_t *smem) {
  return batched_staged_any<float, float>(tile_y, stages, blocks_per_sm, self_on, t1, smem);
}
cudaError_t scgb::staged_occupancy_f32(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                       int *blocks) {
  return staged_occupancy<float, float>(tile_y, stages, blocks_per_sm, self_on, t1, blocks);
}
cudaError_t scgb::generic_occupancy_f32(int lattice, int stencil, int tile_y, bool t1, int *blocks) {
  return generic_occupancy<float, float>(lattice, stencil, tile_y, t1, blocks);
}
const void *scgb::persistent_staged_kernel_f32(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                              size_t *smem) {
  return persistent_staged_any<float, float>(tile_y, stages, blocks_per_sm, self_on, t1, smem);
}

__global__ void scgb::grid_barrier_probe(unsigned *counter, unsigned *err, unsigned max_polls) {
  if (!grid_step_barrier(counter, 2u, max_polls) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(err, 2u);
}
cudaError_t scgb::launch_barrier_probe(unsigned *counter, unsigned *err, unsigned max_polls, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  grid_barrier_probe<<<1, 32, 0, st>>>(counter, err, max_polls);
  return cudaGetLastError();
}
