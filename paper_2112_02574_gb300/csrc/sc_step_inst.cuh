// Instantiation helper: included by one translation unit per storage type
// (so the four instantiation sets compile in parallel).
#pragma once

#include "sc_dispatch.h"
#include "sc_step_kernel.cuh"

namespace scgb {

template <int LAT, int STEN, class ST, class CT, int TY>
cudaError_t launch_one(const StepLaunch &l, const StepArgs<CT> &a) {
  constexpr size_t smem = step_smem_bytes<LAT, STEN, CT, TY>();
  auto *k = sc_step_kernel<LAT, STEN, ST, CT, TY>;
  static bool attr_set = false;  // the attribute is per function; set it once
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k<<<l.grid, dim3(32, TY), smem, l.stream>>>(a);
  return cudaGetLastError();
}

template <int LAT, int STEN, class ST, class CT>
cudaError_t launch_ty(const StepLaunch &l, const StepArgs<CT> &a) {
  switch (l.tile_y) {
    case 1: return launch_one<LAT, STEN, ST, CT, 1>(l, a);
    case 2: return launch_one<LAT, STEN, ST, CT, 2>(l, a);
    case 4: return launch_one<LAT, STEN, ST, CT, 4>(l, a);
    case 8: return launch_one<LAT, STEN, ST, CT, 8>(l, a);
    default: return cudaErrorInvalidValue;
  }
}

template <class ST, class CT>
cudaError_t launch_any(const StepLaunch &l, const StepArgs<CT> &a) {
  if (l.lattice == kD3Q19 && l.stencil == kE4) return launch_ty<kD3Q19, kE4, ST, CT>(l, a);
  if (l.lattice == kD3Q19 && l.stencil == kE6) return launch_ty<kD3Q19, kE6, ST, CT>(l, a);
  if (l.lattice == kD2Q9 && l.stencil == kE4) return launch_ty<kD2Q9, kE4, ST, CT>(l, a);
  return cudaErrorInvalidValue;
}

}  // namespace scgb
