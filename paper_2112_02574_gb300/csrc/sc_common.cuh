// Device-side building blocks shared by the kernels of this library:
// velocity sets, forcing stencils, component-pair arithmetic, storage codecs
// and kernel argument structs.
//
// Model: two-component Shan-Chen lattice Boltzmann method of arXiv:2112.02574,
// section 2 (Eqs. lbm, omega_i, Guo, feq, u, sc_force), c_s^2 = 1/3.
//
// Population storage is component-interleaved: the value of component J in
// direction i at site s sits at element (i * N + s) * 2 + J, so one access
// carries both components of a direction and site (8 bytes in FP32), and the
// two components are computed together with paired (FP32x2) arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/sc.h"

namespace scgb {

constexpr int kD2Q9 = 0, kD3Q19 = 1;

// ------------------------------------------------------------ arithmetic
// Explicitly rounded arithmetic: the step kernels spell every operation of the
// collision with these, so kernels of different shape produce bitwise identical
// results whatever the compiler would otherwise contract.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float expm1_ct(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_ct(double x) { return expm1(x); }

// Component pairs (x = A, y = B).  FP32 pairs use the packed FP32x2 operations
// of sm_100+ (each lane rounded exactly like its scalar counterpart).
template <class CT>
struct Pair;
template <>
struct Pair<float> {
  using T = float2;
};
template <>
struct Pair<double> {
  using T = double2;
};
template <class CT>
using P2 = typename Pair<CT>::T;

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pset(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pbc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 pswap(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(radd(a.x, b.x), radd(a.y, b.y)); }
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(rsub(a.x, b.x), rsub(a.y, b.y)); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(rmul(a.x, b.x), rmul(a.y, b.y)); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(rfma(a.x, b.x, c.x), rfma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 pset(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ double2 pbc(double s) { return make_double2(s, s); }
__device__ __forceinline__ double2 pswap(double2 a) { return make_double2(a.y, a.x); }

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
// A component pair (A, B) of one direction and site: stored -> compute pair and
// back.  F16 carries a per-component power-of-two scale that puts the
// deviations high in the normal range (a power of two changes no rounding of a
// normal FP16 number, only how far the values sit from underflow and overflow);
// BF16 has the FP32 exponent range and needs none.  SMEM selects plain loads
// (shared memory) instead of read-only-cache loads (global memory).
template <class ST, class CT>
struct Codec2;
template <>
struct Codec2<float, float> {
  template <bool SMEM>
  __device__ __forceinline__ static float2 load(const float *p, float2) {
    return SMEM ? *reinterpret_cast<const float2 *>(p) : __ldg(reinterpret_cast<const float2 *>(p));
  }
  __device__ __forceinline__ static void store(float *p, float2 v, float2) { *reinterpret_cast<float2 *>(p) = v; }
};
template <>
struct Codec2<double, double> {
  template <bool SMEM>
  __device__ __forceinline__ static double2 load(const double *p, double2) {
    return SMEM ? *reinterpret_cast<const double2 *>(p) : __ldg(reinterpret_cast<const double2 *>(p));
  }
  __device__ __forceinline__ static void store(double *p, double2 v, double2) {
    *reinterpret_cast<double2 *>(p) = v;
  }
};
// F16 pairs are read and written in scaled units (see scaled_units below): the step
// arithmetic itself carries the power-of-two scale, so no multiply happens here.
template <>
struct Codec2<__half, float> {
  template <bool SMEM>
  __device__ __forceinline__ static float2 load(const __half *p, float2) {
    const __half2 h = SMEM ? *reinterpret_cast<const __half2 *>(p) : __ldg(reinterpret_cast<const __half2 *>(p));
    return __half22float2(h);
  }
  __device__ __forceinline__ static void store(__half *p, float2 v, float2) {
    *reinterpret_cast<__half2 *>(p) = __float22half2_rn(v);
  }
};
template <>
struct Codec2<__nv_bfloat16, float> {
  template <bool SMEM>
  __device__ __forceinline__ static float2 load(const __nv_bfloat16 *p, float2) {
    const __nv_bfloat162 h =
        SMEM ? *reinterpret_cast<const __nv_bfloat162 *>(p) : __ldg(reinterpret_cast<const __nv_bfloat162 *>(p));
    return __bfloat1622float2(h);
  }
  __device__ __forceinline__ static void store(__nv_bfloat16 *p, float2 v, float2) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(v);
  }
};

// Units of the step arithmetic.  F16 storage keeps its values multiplied by a
// power-of-two scale 2^k(J) per component; its step computes the population
// pairs in those scaled units directly (the weights w_i enter as w_i 2^k, sums
// and momenta are scaled back once), which saves a multiply per population read
// and per population written.  A power of two commutes with every rounding (no
// value is near the FP32 range limits), so the results are bit for bit those of
// the same arithmetic on unscaled values.  Every other storage computes on the
// values themselves.
template <class ST>
__host__ __device__ constexpr bool scaled_units() {
  return std::is_same<ST, __half>::value;
}

// ---------------------------------------------------------------- arguments
template <class CT>
struct StepArgs {
  const void *src;  // populations (post-collision of the previous step, stored at the collision site)
  void *dst;
  int nx, ny, nz, tile_z;
  int64_t N;         // sites
  P2<CT> nbar;       // storage reference densities (A, B)
  P2<CT> omega;      // 1 / tau_J
  P2<CT> guo;        // 1 - 1 / (2 tau_J)
  CT gcross;         // -G c_s^2
  P2<CT> gself;      // -G_JJ c_s^2
  P2<CT> psibar;     // psi(nbar_J)
  int self_on;       // any G_JJ != 0
  int tau_one;       // tau_A = tau_B = 1: the relaxation keeps nothing of f (see carry_size)
  int psi_exp;       // psi = exp(-1/n) (else psi = n)
  P2<CT> scale;      // storage scale 2^k(J) (F16; unused for the other storages)
  P2<CT> inv_scale;  // 2^-k(J)
  unsigned int *err;     // device status word (bit 0: density out of range)
  // Local reference (F16/BF16 storage): the value stored at site s is
  // (f*_i(s) - w_i n(s)) 2^k with n(s) the site's density when it was written;
  // n(s) - nbar is kept as an FP32 pair per site: read from nsrc, written to ndst.
  const float2 *nsrc;
  float2 *ndst;
  // Balanced z split of a single-lattice step launch (zbal_k > 0; 1-D grid of
  // zbal_k * zbal_cols + zbal_rem blocks): zbal_cols = x tiles * y tiles, zbal_cols_x = x tiles.
  int zbal_k, zbal_rem, zbal_cols, zbal_cols_x;
};

// Storage modes whose populations are deviations from each site's own density
// (16-bit storage); the 32/64-bit modes use the constant mean density nbar.
template <class ST>
__host__ __device__ constexpr bool local_ref() {
  return sizeof(ST) == 2;
}

__host__ __device__ __forceinline__ int wrapi(int a, int n) {
  // a in [-n, 2n)
  return a < 0 ? a + n : (a >= n ? a - n : a);
}

}  // namespace scgb
