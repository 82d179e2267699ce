// Device-side building blocks shared by the kernels of this library:
// velocity sets, forcing stencils, storage codecs and kernel argument structs.
//
// Model: two-component Shan-Chen lattice Boltzmann method of arXiv:2112.02574,
// section 2 (Eqs. lbm, omega_i, Guo, feq, u, sc_force), c_s^2 = 1/3.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sc.h"

namespace scgb {

constexpr int kD2Q9 = 0, kD3Q19 = 1;

// ---------------------------------------------------------------- lattices
// D3Q19 velocities, opposite directions adjacent (the order sc.h documents).
__host__ __device__ constexpr int d3q19_c(int i, int d) {
  constexpr int c[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                            {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                            {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
  return c[i][d];
}
__host__ __device__ constexpr int d2q9_c(int i, int d) {
  constexpr int c[9][3] = {{0, 0, 0}, {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                           {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
  return c[i][d];
}

template <int LAT>
struct Lattice;

template <>
struct Lattice<kD3Q19> {
  static constexpr int Q = 19;
  static constexpr int DIM = 3;
  __host__ __device__ static constexpr int c(int i, int d) { return d3q19_c(i, d); }
  // w_i = 1/3, 1/18, 1/36 by |c|^2 (W = w / c_s^2 gives the 1/6, 1/12 of Eq. sc_force)
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
};

template <>
struct Lattice<kD2Q9> {
  static constexpr int Q = 9;
  static constexpr int DIM = 2;
  __host__ __device__ static constexpr int c(int i, int d) { return d2q9_c(i, d); }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
};

// ---------------------------------------------------------------- stencils
// Half forcing stencils: one vector per +/- pair, with W(|v|^2).
//   E4 on D3Q19: 9 vectors, W(1) = 1/6, W(2) = 1/12 (section 2);
//   E4 on D2Q9 : 4 vectors, W(1) = 1/3, W(2) = 1/12;
//   E6 on D3Q19: 16 vectors on shells |v|^2 = 1, 2, 3, 4 with
//                W = 2/15, 1/15, 1/60, 1/120 (4th- and 6th-order isotropy, e_2 = 1).
__host__ __device__ constexpr int e4_3d_v(int a, int d) {
  constexpr int v[9][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0},
                           {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
  return v[a][d];
}
__host__ __device__ constexpr int e4_2d_v(int a, int d) {
  constexpr int v[4][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {1, -1, 0}};
  return v[a][d];
}
__host__ __device__ constexpr int e6_v(int a, int d) {
  constexpr int v[16][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},  {1, -1, 0}, {1, 0, 1},
                            {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},  {1, 1, -1}, {1, -1, 1},
                            {1, -1, -1}, {2, 0, 0}, {0, 2, 0},  {0, 0, 2}};
  return v[a][d];
}

constexpr int kE4 = 0, kE6 = 1;

template <int LAT, int STEN>
struct Stencil;

template <>
struct Stencil<kD3Q19, kE4> {
  static constexpr int NH = 9;     // half-stencil size
  static constexpr int HALO = 1;   // reach in lattice units
  __host__ __device__ static constexpr int v(int a, int d) { return e4_3d_v(a, d); }
  __host__ __device__ static constexpr double W(int a) { return a < 3 ? 1.0 / 6.0 : 1.0 / 12.0; }
};
template <>
struct Stencil<kD2Q9, kE4> {
  static constexpr int NH = 4;
  static constexpr int HALO = 1;
  __host__ __device__ static constexpr int v(int a, int d) { return e4_2d_v(a, d); }
  __host__ __device__ static constexpr double W(int a) { return a < 2 ? 1.0 / 3.0 : 1.0 / 12.0; }
};
template <>
struct Stencil<kD3Q19, kE6> {
  static constexpr int NH = 16;
  static constexpr int HALO = 2;
  __host__ __device__ static constexpr int v(int a, int d) { return e6_v(a, d); }
  __host__ __device__ static constexpr double W(int a) {
    return a < 3 ? 2.0 / 15.0 : (a < 9 ? 1.0 / 15.0 : (a < 13 ? 1.0 / 60.0 : 1.0 / 120.0));
  }
};

// ---------------------------------------------------------------- storage
// Stored value -> compute type and back.  F16/BF16 carry a per-(J, i)
// power-of-two scale so that the deviations sit in the normal range.
template <class S, class CT>
struct Codec {
  __device__ __forceinline__ static CT load(const S *p, CT /*inv_scale*/) { return CT(__ldg(p)); }
  __device__ __forceinline__ static void store(S *p, CT v, CT /*scale*/) { *p = S(v); }
};
template <>
struct Codec<__half, float> {
  __device__ __forceinline__ static float load(const __half *p, float inv_scale) {
    return __half2float(__ldg(p)) * inv_scale;
  }
  __device__ __forceinline__ static void store(__half *p, float v, float scale) { *p = __float2half_rn(v * scale); }
};
template <>
struct Codec<__nv_bfloat16, float> {
  __device__ __forceinline__ static float load(const __nv_bfloat16 *p, float inv_scale) {
    return __bfloat162float(__ldg(p)) * inv_scale;
  }
  __device__ __forceinline__ static void store(__nv_bfloat16 *p, float v, float scale) {
    *p = __float2bfloat16_rn(v * scale);
  }
};

// ---------------------------------------------------------------- arguments
template <class CT>
struct StepArgs {
  const void *src;  // populations (post-collision of the previous step, stored at the collision site)
  void *dst;
  int nx, ny, nz, tile_z;
  int64_t N;        // sites = plane stride
  CT nbar[2];       // storage reference densities
  CT omega[2];      // 1 / tau_J
  CT guo[2];        // 1 - 1 / (2 tau_J)
  CT gcross;        // -G c_s^2
  CT gself[2];      // -G_JJ c_s^2
  CT psibar[2];     // psi(nbar_J)
  int self_on;      // any G_JJ != 0
  int psi_exp;      // psi = exp(-1/n) (else psi = n)
  CT scale[2][19];      // storage scale 2^k (1 for F32/F64)
  CT inv_scale[2][19];  // 2^-k
  unsigned int *err;    // device status word (bit 0: non-positive density)
};

__device__ __forceinline__ float expm1_ct(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_ct(double x) { return expm1(x); }

__host__ __device__ __forceinline__ int wrapi(int a, int n) {
  // a in [-n, 2n)
  return a < 0 ? a + n : (a >= n ? a - n : a);
}

}  // namespace scgb
