// Instantiation helper: included by one translation unit per storage type
// (so the four instantiation sets compile in parallel).
#pragma once

#include <mutex>
#include <set>
#include <type_traits>
#include <utility>

#include "sc_dispatch.h"
#include "sc_step_kernel.cuh"
#include "sc_step_staged.cuh"

namespace scgb {

// Set a kernel's dynamic shared-memory limit once per device (the attribute belongs to
// the function on the current device); false (with the CUDA error pending) on failure.
inline bool attr_once(const void *k, size_t smem) {
  static std::mutex m;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(m);
  if (done.count({k, dev})) return true;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) return false;
  done.insert({k, dev});
  return true;
}

// T1 selects the tau_A = tau_B = 1 instantiation (StepArgs::tau_one).
template <int LAT, int STEN, class ST, class CT, int TY>
cudaError_t launch_one(const StepLaunch &l, const StepArgs<CT> &a) {
  constexpr size_t smem = step_smem_bytes<LAT, STEN, CT, TY>();
  auto *k = a.tau_one ? sc_step_kernel<LAT, STEN, ST, CT, TY, true> : sc_step_kernel<LAT, STEN, ST, CT, TY, false>;
  if (!attr_once(reinterpret_cast<const void *>(k), smem)) return cudaGetLastError();
  const dim3 grid = a.zbal_k > 0 ? dim3(a.zbal_k * a.zbal_cols + a.zbal_rem) : l.grid;
  k<<<grid, dim3(32, TY), smem, l.stream>>>(a);
  return cudaGetLastError();
}

template <int LAT, int STEN, class ST, class CT, int TY>
cudaError_t generic_occupancy_one(bool t1, int *blocks) {
  constexpr size_t smem = step_smem_bytes<LAT, STEN, CT, TY>();
  auto *k = t1 ? sc_step_kernel<LAT, STEN, ST, CT, TY, true> : sc_step_kernel<LAT, STEN, ST, CT, TY, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, 32 * TY, smem);
}

// Resident blocks per SM of the generic kernel for (lattice, stencil, tile_y).
template <class ST, class CT>
cudaError_t generic_occupancy(int lat, int sten, int ty, bool t1, int *blocks) {
  auto by_ty = [&](auto lat_c, auto sten_c) -> cudaError_t {
    constexpr int LAT = decltype(lat_c)::value, STEN = decltype(sten_c)::value;
    switch (ty) {
      case 1: return generic_occupancy_one<LAT, STEN, ST, CT, 1>(t1, blocks);
      case 2: return generic_occupancy_one<LAT, STEN, ST, CT, 2>(t1, blocks);
      case 4: return generic_occupancy_one<LAT, STEN, ST, CT, 4>(t1, blocks);
      case 8: return generic_occupancy_one<LAT, STEN, ST, CT, 8>(t1, blocks);
      default: return cudaErrorInvalidValue;
    }
  };
  if (lat == kD3Q19 && sten == kE4) return by_ty(std::integral_constant<int, kD3Q19>{}, std::integral_constant<int, kE4>{});
  if (lat == kD3Q19 && sten == kE6) return by_ty(std::integral_constant<int, kD3Q19>{}, std::integral_constant<int, kE6>{});
  if (lat == kD2Q9 && sten == kE4) return by_ty(std::integral_constant<int, kD2Q9>{}, std::integral_constant<int, kE4>{});
  return cudaErrorInvalidValue;
}

// Staged kernel: one block per (x column, y column, z chunk), like the generic kernel.
template <class ST, class CT, int TY, int NS, int MINB>
cudaError_t launch_staged_one(const StepLaunch &l, const StepArgs<CT> &a) {
  constexpr size_t smem_max = staged_smem_bytes<ST, CT, TY, NS>();
  const size_t smem = staged_smem_bytes<ST, CT, TY, NS>(a.self_on != 0);
  auto *k = a.tau_one ? sc_step_staged<ST, CT, TY, NS, MINB, true> : sc_step_staged<ST, CT, TY, NS, MINB, false>;
  if (!attr_once(reinterpret_cast<const void *>(k), smem_max)) return cudaGetLastError();
  const dim3 grid = a.zbal_k > 0 ? dim3(a.zbal_k * a.zbal_cols + a.zbal_rem)
                                 : dim3((a.nx + 31) / 32, (a.ny + TY - 1) / TY, (a.nz + a.tile_z - 1) / a.tile_z);
  k<<<grid, dim3(32, TY), smem, l.stream>>>(a);
  return cudaGetLastError();
}

template <class ST, class CT, int TY, int NS, int MINB>
cudaError_t staged_occupancy_one(bool self_on, bool t1, int *blocks) {
  auto *k = t1 ? sc_step_staged<ST, CT, TY, NS, MINB, true> : sc_step_staged<ST, CT, TY, NS, MINB, false>;
  cudaError_t e =
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(staged_smem_bytes<ST, CT, TY, NS>()));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, 32 * TY,
                                                       staged_smem_bytes<ST, CT, TY, NS>(self_on));
}

// One instantiated staged configuration, as a tag type.
template <int TY_, int NS_, int MINB_>
struct StagedCfg {
  static constexpr int TY = TY_, NS = NS_, MINB = MINB_;
};

// Calls fn(StagedCfg<...>{}) for the instantiated configuration (tile_y, stages,
// blocks per SM) that serves the request, or returns fallback.  Instantiated:
// (4, 1|2, 2|3) for every storage; (8, 1|2, 1|2) and (16, 1, 1) except F64;
// (16, 2, 1) for 16-bit storage only (two 32 x 16 FP32 stages do not fit).
// blocks_per_sm below the smallest instantiated value takes that value.
template <class ST, class Fn, class R>
R with_staged_cfg(int ty, int ns, int mb, R fallback, Fn &&fn) {
  if (ty == 4) {
    if (ns == 2 && mb <= 2) return fn(StagedCfg<4, 2, 2>{});
    if (ns == 2 && mb == 3) return fn(StagedCfg<4, 2, 3>{});
    if (ns == 1 && mb <= 2) return fn(StagedCfg<4, 1, 2>{});
    if (ns == 1 && mb == 3) return fn(StagedCfg<4, 1, 3>{});
  }
  if constexpr (sizeof(ST) < 8) {
    if (ty == 8) {
      if (ns == 2 && mb <= 1) return fn(StagedCfg<8, 2, 1>{});
      if (ns == 2 && mb == 2) return fn(StagedCfg<8, 2, 2>{});
      if (ns == 1 && mb <= 1) return fn(StagedCfg<8, 1, 1>{});
      if (ns == 1 && mb == 2) return fn(StagedCfg<8, 1, 2>{});
      if (ns == 1 && mb == 3) return fn(StagedCfg<8, 1, 3>{});
    }
    if (ty == 16 && mb <= 1) {
      if (ns == 1) return fn(StagedCfg<16, 1, 1>{});
      if constexpr (sizeof(ST) == 2) {
        if (ns == 2) return fn(StagedCfg<16, 2, 1>{});
      }
    }
  }
  return fallback;
}

// Resident blocks per SM of the staged kernel for (tile_y, stages, blocks_per_sm).
template <class ST, class CT>
cudaError_t staged_occupancy(int ty, int ns, int mb, bool self_on, bool t1, int *blocks) {
  return with_staged_cfg<ST>(ty, ns, mb, cudaErrorInvalidValue, [&](auto cfg) {
    using C = decltype(cfg);
    return staged_occupancy_one<ST, CT, C::TY, C::NS, C::MINB>(self_on, t1, blocks);
  });
}

template <class ST, class CT>
cudaError_t launch_staged(const StepLaunch &l, const StepArgs<CT> &a) {
  if (l.lattice != kD3Q19 || l.stencil != kE4 || a.nx < 32 || a.nx % StagedGeom<ST, 4>::CE != 0)
    return cudaErrorInvalidValue;
  return with_staged_cfg<ST>(l.tile_y, l.stages, l.blocks_per_sm, cudaErrorInvalidValue, [&](auto cfg) {
    using C = decltype(cfg);
    return launch_staged_one<ST, CT, C::TY, C::NS, C::MINB>(l, a);
  });
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
  if (l.staged) return launch_staged<ST, CT>(l, a);
  if (l.lattice == kD3Q19 && l.stencil == kE4) return launch_ty<kD3Q19, kE4, ST, CT>(l, a);
  if (l.lattice == kD3Q19 && l.stencil == kE6) return launch_ty<kD3Q19, kE6, ST, CT>(l, a);
  if (l.lattice == kD2Q9 && l.stencil == kE4) return launch_ty<kD2Q9, kE4, ST, CT>(l, a);
  return cudaErrorInvalidValue;
}

template <int LAT, int STEN, class ST, class CT, int TY>
const void *batched_one(bool t1, size_t *smem) {
  constexpr size_t bytes = step_smem_bytes<LAT, STEN, CT, TY>();
  auto *k = t1 ? sc_step_batched<LAT, STEN, ST, CT, TY, true> : sc_step_batched<LAT, STEN, ST, CT, TY, false>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)) != cudaSuccess) return nullptr;
  *smem = bytes;
  return reinterpret_cast<const void *>(k);
}

template <int LAT, int STEN, class ST, class CT>
const void *batched_ty(int ty, bool t1, size_t *smem) {
  switch (ty) {
    case 1: return batched_one<LAT, STEN, ST, CT, 1>(t1, smem);
    case 2: return batched_one<LAT, STEN, ST, CT, 2>(t1, smem);
    case 4: return batched_one<LAT, STEN, ST, CT, 4>(t1, smem);
    case 8: return batched_one<LAT, STEN, ST, CT, 8>(t1, smem);
    default: return nullptr;
  }
}

template <class ST, class CT>
const void *batched_any(int lat, int sten, int ty, bool t1, size_t *smem) {
  if (lat == kD3Q19 && sten == kE4) return batched_ty<kD3Q19, kE4, ST, CT>(ty, t1, smem);
  if (lat == kD3Q19 && sten == kE6) return batched_ty<kD3Q19, kE6, ST, CT>(ty, t1, smem);
  if (lat == kD2Q9 && sten == kE4) return batched_ty<kD2Q9, kE4, ST, CT>(ty, t1, smem);
  return nullptr;
}

template <class ST, class CT, int TY, int NS, int MINB>
const void *batched_staged_one(bool self_on, bool t1, size_t *smem) {
  auto *k = t1 ? sc_step_staged_batched<ST, CT, TY, NS, MINB, true> : sc_step_staged_batched<ST, CT, TY, NS, MINB, false>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(staged_smem_bytes<ST, CT, TY, NS>())) != cudaSuccess)
    return nullptr;
  *smem = staged_smem_bytes<ST, CT, TY, NS>(self_on);
  return reinterpret_cast<const void *>(k);
}

template <class ST, class CT, int TY, int NS, int MINB>
const void *persistent_staged_one(bool self_on, bool t1, size_t *smem) {
  auto *k = t1 ? sc_step_staged_persistent<ST, CT, TY, NS, MINB, true>
               : sc_step_staged_persistent<ST, CT, TY, NS, MINB, false>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(staged_smem_bytes<ST, CT, TY, NS>())) != cudaSuccess)
    return nullptr;
  *smem = staged_smem_bytes<ST, CT, TY, NS>(self_on);
  return reinterpret_cast<const void *>(k);
}

// Same configurations as launch_staged.
template <class ST, class CT>
const void *persistent_staged_any(int ty, int ns, int mb, bool self_on, bool t1, size_t *smem) {
  return with_staged_cfg<ST>(ty, ns, mb, static_cast<const void *>(nullptr), [&](auto cfg) {
    using C = decltype(cfg);
    return persistent_staged_one<ST, CT, C::TY, C::NS, C::MINB>(self_on, t1, smem);
  });
}

// Same configurations as launch_staged.
template <class ST, class CT>
const void *batched_staged_any(int ty, int ns, int mb, bool self_on, bool t1, size_t *smem) {
  return with_staged_cfg<ST>(ty, ns, mb, static_cast<const void *>(nullptr), [&](auto cfg) {
    using C = decltype(cfg);
    return batched_staged_one<ST, CT, C::TY, C::NS, C::MINB>(self_on, t1, smem);
  });
}

}  // namespace scgb
