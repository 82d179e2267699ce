// Host-side entry points of the per-storage kernel instantiation units.
#pragma once

#include <cuda_runtime.h>

#include "sc_common.cuh"

namespace scgb {

struct StepLaunch {
  int lattice;  // kD2Q9 / kD3Q19
  int stencil;  // kE4 / kE6
  int tile_y;   // 1, 2, 4 or 8
  int staged;   // 1: cp.async-staged kernel (D3Q19, E4, nx >= 32, nx a multiple of the chunk sites)
  int stages;   // staged kernel: pipeline stages, 1 or 2
  int blocks_per_sm;  // staged kernel: resident blocks per SM its registers allow (tile_y 4: 2 or 3; 8: 1 or 2)
  dim3 grid;    // generic kernel grid without a balanced z split
  cudaStream_t stream;
};

// Launch one fused time step; returns the launch error (cudaErrorInvalidValue
// for an unsupported lattice / stencil / tile combination).
cudaError_t launch_step_f32(const StepLaunch &l, const StepArgs<float> &a);
cudaError_t launch_step_f16(const StepLaunch &l, const StepArgs<float> &a);
cudaError_t launch_step_bf16(const StepLaunch &l, const StepArgs<float> &a);
cudaError_t launch_step_f64(const StepLaunch &l, const StepArgs<double> &a);

// The batched step kernel for one (lattice, stencil, tile_y) combination, as a
// function pointer for graph kernel nodes (nullptr if unsupported); *smem
// receives its dynamic shared-memory bytes.  Parameters: (const StepArgs *args,
// const int4 *items, int swap), block (32, tile_y), one block per item.  t1: every
// member has tau_A = tau_B = 1 (the instantiation that carries momentum sums only).
const void *batched_kernel_f32(int lattice, int stencil, int tile_y, bool t1, size_t *smem);
const void *batched_kernel_f16(int lattice, int stencil, int tile_y, bool t1, size_t *smem);
const void *batched_kernel_bf16(int lattice, int stencil, int tile_y, bool t1, size_t *smem);
const void *batched_kernel_f64(int lattice, int stencil, int tile_y, bool t1, size_t *smem);

// Resident blocks per SM of the staged step kernel for (tile_y, stages, blocks_per_sm),
// with or without the psi ring of a self coupling.
cudaError_t staged_occupancy_f32(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1, int *blocks);
cudaError_t staged_occupancy_f16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1, int *blocks);
cudaError_t staged_occupancy_bf16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1, int *blocks);
cudaError_t staged_occupancy_f64(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1, int *blocks);

// Resident blocks per SM of the generic step kernel for (lattice, stencil, tile_y).
cudaError_t generic_occupancy_f32(int lattice, int stencil, int tile_y, bool t1, int *blocks);
cudaError_t generic_occupancy_f16(int lattice, int stencil, int tile_y, bool t1, int *blocks);
cudaError_t generic_occupancy_bf16(int lattice, int stencil, int tile_y, bool t1, int *blocks);
cudaError_t generic_occupancy_f64(int lattice, int stencil, int tile_y, bool t1, int *blocks);

// The batched staged step kernel (D3Q19, E4) for (tile_y, stages, blocks_per_sm),
// same parameters and block shape as above; nullptr if not instantiated.  self_on:
// some member has a self coupling (the psi ring is then part of *smem).
const void *batched_staged_kernel_f32(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                         size_t *smem);
const void *batched_staged_kernel_f16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                         size_t *smem);
const void *batched_staged_kernel_bf16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                         size_t *smem);
const void *batched_staged_kernel_f64(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                         size_t *smem);

// The persistent batched staged step kernel (D3Q19, E4), same configurations: parameters
// (const StepArgs *args, const int4 *items, int nitems, int nsteps, int swap0, unsigned *counter,
// int nlat), block (32, tile_y), launched cooperatively with at most the co-resident blocks;
// nullptr if not instantiated.
const void *persistent_staged_kernel_f32(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                         size_t *smem);
const void *persistent_staged_kernel_f16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                         size_t *smem);
const void *persistent_staged_kernel_bf16(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                          size_t *smem);
const void *persistent_staged_kernel_f64(int tile_y, int stages, int blocks_per_sm, bool self_on, bool t1,
                                         size_t *smem);
// Self-test of the persistent launch's bounded grid-barrier wait (one block, a barrier that never
// completes): zeroes *counter, then the wait runs out after max_polls polls and sets bit 1 of *err.
cudaError_t launch_barrier_probe(unsigned *counter, unsigned *err, unsigned max_polls, cudaStream_t st);

}  // namespace scgb
