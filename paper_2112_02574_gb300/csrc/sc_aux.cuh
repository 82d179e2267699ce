// Kernels around the time step: initial state, population access, FP64
// density / pseudopotential fields, the common velocity, the lattice pressure
// tensor with its profiles, the sigma[R] minimum and conserved totals.
// All analysis arithmetic is FP64 (arXiv:2112.02574, sections 2 and 3).
#pragma once

#include "sc_common.cuh"
#include "sc_profile.cuh"

namespace scgb {

// Storage read / write in FP64 (natural populations f = g / scale + w nbar).
// Populations are component-interleaved: element (i * N + s) * 2 + J.
__device__ __forceinline__ double to_double(float v) { return v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(__half v) { return __half2float(v); }
__device__ __forceinline__ double to_double(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class ST>
__device__ __forceinline__ ST from_double(double v);
template <>
__device__ __forceinline__ float from_double<float>(double v) { return float(v); }
template <>
__device__ __forceinline__ double from_double<double>(double v) { return v; }
template <>
__device__ __forceinline__ __half from_double<__half>(double v) { return __float2half_rn(float(v)); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn(float(v));
}
template <class ST>
__device__ __forceinline__ double load_dev(const ST *p, double inv_scale) {
  return to_double(*p) * inv_scale;
}
template <class ST>
__device__ __forceinline__ void store_dev(ST *p, double v, double scale) {
  *p = from_double<ST>(v * scale);
}

struct PopArgs {
  void *buf;         // stored populations [Q][N][2]
  float2 *nref;      // local reference density deviations n_ref - nbar [N] (16-bit storage; nullptr otherwise)
  int nx, ny, nz;
  int64_t N;
  double nbar[2];
  double scale[2][19];
  double inv_scale[2][19];
};

// Natural FP64 population of direction i, component J stored at site s.
template <int LAT, class ST>
__device__ __forceinline__ double pop_value(const PopArgs &a, const ST *buf, int i, int J, int64_t s) {
  const double g = load_dev<ST>(buf + ((int64_t)i * a.N + s) * 2 + J, a.inv_scale[J][i]);
  const double ref = a.nbar[J] + (local_ref<ST>() ? double(J == 0 ? a.nref[s].x : a.nref[s].y) : 0.0);
  return g + Lattice<LAT>::w(i) * ref;
}

// mode 0: initial rest equilibrium from densities n0 (FP64 [2][N]): the value
//         stored at y for direction i is w_i n0_J(y + xi_i), so that the first
//         pull delivers f_i(x) = w_i n0_J(x);
// mode 1: natural populations f (FP64 [2][Q][N]) -> storage (inverse pull);
// mode 2: storage -> natural populations f.
// Stored values are relative to w_i nbar_J, or with a local reference to
// w_i nref_J(y) where nref(y) is the sum of the values stored at y.
template <int LAT, class ST>
__global__ void pop_kernel(PopArgs a, int mode, const double *n0A, const double *n0B, double *f) {
  using L = Lattice<LAT>;
  ST *buf = static_cast<ST *>(a.buf);
  const int64_t N = a.N;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords(s, a.nx, a.ny, x, y, z);
    if (mode == 2) {
#pragma unroll
      for (int J = 0; J < 2; ++J)
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          const int64_t bwd = site_at(x - L::c(i, 0), y - L::c(i, 1), z - L::c(i, 2), a.nx, a.ny, a.nz);
          f[((int64_t)J * L::Q + i) * N + s] = pop_value<LAT, ST>(a, buf, i, J, bwd);
        }
      continue;
    }
    double ref[2];
#pragma unroll
    for (int J = 0; J < 2; ++J) {
      if constexpr (local_ref<ST>()) {
        double sum = 0.0;
        if (mode == 0) {
          sum = (J == 0 ? n0A : n0B)[s];
        } else {
#pragma unroll
          for (int i = 0; i < L::Q; ++i)
            sum += f[((int64_t)J * L::Q + i) * N + site_at(x + L::c(i, 0), y + L::c(i, 1), z + L::c(i, 2), a.nx, a.ny, a.nz)];
        }
        ref[J] = a.nbar[J] + double(float(sum - a.nbar[J]));  // the deviation is kept in FP32
      } else {
        ref[J] = a.nbar[J];
      }
    }
    if constexpr (local_ref<ST>())
      a.nref[s] = make_float2(float(ref[0] - a.nbar[0]), float(ref[1] - a.nbar[1]));
#pragma unroll
    for (int J = 0; J < 2; ++J)
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const double w = L::w(i);
        const int64_t fwd = site_at(x + L::c(i, 0), y + L::c(i, 1), z + L::c(i, 2), a.nx, a.ny, a.nz);
        const double v = mode == 0 ? w * (J == 0 ? n0A : n0B)[fwd] : f[((int64_t)J * L::Q + i) * N + fwd];
        store_dev<ST>(buf + ((int64_t)i * N + s) * 2 + J, v - w * ref[J], a.scale[J][i]);
      }
  }
}

// FP64 density fields n_J (and psi_J) from the stored state (pull + sum).
// fields: [4][N] = n_A, n_B, psi_A, psi_B.
template <int LAT, class ST>
__global__ void fields_kernel(PopArgs a, int psi_exp, double *fields) {
  using L = Lattice<LAT>;
  const ST *buf = static_cast<const ST *>(a.buf);
  const int64_t N = a.N;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords(s, a.nx, a.ny, x, y, z);
#pragma unroll
    for (int J = 0; J < 2; ++J) {
      double n = 0.0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const int64_t bwd = site_at(x - L::c(i, 0), y - L::c(i, 1), z - L::c(i, 2), a.nx, a.ny, a.nz);
        n += pop_value<LAT, ST>(a, buf, i, J, bwd);
      }
      fields[J * N + s] = n;
      fields[(2 + J) * N + s] = psi_exp ? exp(-1.0 / n) : n;
    }
  }
}


// Eq. sc_force at site s from FP64 fields, +/- pairs first.
template <int LAT, int STEN>
__device__ __forceinline__ void force64(const ForceParams &p, const double *fields, int x, int y, int z, int64_t s,
                                        double F[2][3]) {
  using SN = Stencil<LAT, STEN>;
  const double cs2 = 1.0 / 3.0;
  double S[2][3] = {{0, 0, 0}, {0, 0, 0}}, T[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int k = 0; k < SN::NH; ++k) {
    const int v0 = SN::v(k, 0), v1 = SN::v(k, 1), v2 = SN::v(k, 2);
    const int64_t sp = site_at(x + v0, y + v1, z + v2, p.nx, p.ny, p.nz);
    const int64_t sm = site_at(x - v0, y - v1, z - v2, p.nx, p.ny, p.nz);
    const double W = SN::W(k);
    const int v[3] = {v0, v1, v2};
#pragma unroll
    for (int J = 0; J < 2; ++J) {
      const double d = fields[J * p.N + sp] - fields[J * p.N + sm];
      const double e = fields[(2 + J) * p.N + sp] - fields[(2 + J) * p.N + sm];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        S[J][m] += W * v[m] * d;
        T[J][m] += W * v[m] * e;
      }
    }
  }
#pragma unroll
  for (int J = 0; J < 2; ++J)
#pragma unroll
    for (int m = 0; m < 3; ++m)
      F[J][m] = -p.G * cs2 * fields[J * p.N + s] * S[1 - J][m] -
                p.G_self[J] * cs2 * fields[(2 + J) * p.N + s] * T[J][m];
}

// Common velocity of Eq. u (force included), FP64 [3][N].
template <int LAT, int STEN, class ST>
__device__ __forceinline__ void site_velocity(const PopArgs &a, const ForceParams &fp, const double *fields,
                                              int64_t s, double u[3]) {
  using L = Lattice<LAT>;
  const ST *buf = static_cast<const ST *>(a.buf);
  const int64_t N = a.N;
  int x, y, z;
  coords(s, a.nx, a.ny, x, y, z);
  double F[2][3];
  force64<LAT, STEN>(fp, fields, x, y, z, s, F);
  double j[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int J = 0; J < 2; ++J)
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int64_t bwd = site_at(x - L::c(i, 0), y - L::c(i, 1), z - L::c(i, 2), a.nx, a.ny, a.nz);
      const double g = pop_value<LAT, ST>(a, buf, i, J, bwd);
#pragma unroll
      for (int m = 0; m < 3; ++m) j[J][m] += L::c(i, m) * g;
    }
  const double n = fields[s] + fields[N + s];
#pragma unroll
  for (int m = 0; m < 3; ++m) u[m] = ((j[0][m] + 0.5 * F[0][m]) + (j[1][m] + 0.5 * F[1][m])) / n;
}

template <int LAT, int STEN, class ST>
__global__ void velocity_kernel(PopArgs a, ForceParams fp, const double *fields, double *u) {
  const int64_t N = a.N;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    double v[3];
    site_velocity<LAT, STEN, ST>(a, fp, fields, s, v);
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m * N + s] = v[m];
  }
}

// Convergence measure of section 4 (criterion on the velocity field): per-block
// partial sums of sum_alpha |u_alpha(x) - u_prev_alpha(x)| over the sites (fixed
// grid-stride order, fixed tree); u_prev is overwritten with u.
template <int LAT, int STEN, class ST>
__global__ void __launch_bounds__(256) velocity_change_partial_kernel(PopArgs a, ForceParams fp, const double *fields,
                                                                      double *u_prev, double *partial) {
  const int64_t N = a.N;
  double acc = 0.0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    double v[3];
    site_velocity<LAT, STEN, ST>(a, fp, fields, s, v);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      acc += fabs(v[m] - u_prev[m * N + s]);
      u_prev[m * N + s] = v[m];
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Centre of mass of one density field's excess over a background value, partial
// sums (w x, w y, w z, w) with w = n(x) - background, in lattice coordinates.
__global__ void __launch_bounds__(256) com_partial_kernel(const double *n, int nx, int ny, int64_t N, double bg,
                                                          double *partial) {
  double acc[4] = {0, 0, 0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords(s, nx, ny, x, y, z);
    const double w = n[s] - bg;
    acc[0] += w * x;
    acc[1] += w * y;
    acc[2] += w * z;
    acc[3] += w;
  }
  __shared__ double red[4][256];
#pragma unroll
  for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) partial[blockIdx.x * 4 + c] = red[c][0];
}

// Block-order finalisation of the two reductions above: kind 0 -> out[0] = scale * sum;
// kind 1 -> out = (X, Y, Z, M) with M the summed weight and X = sum w x / M.
__global__ void finalize_measure_kernel(const double *partial, int nblocks, int kind, double scale, double *out) {
  if (threadIdx.x != 0) return;
  if (kind == 0) {
    double acc = 0.0;
    for (int k = 0; k < nblocks; ++k) acc += partial[k];
    out[0] = scale * acc;
    return;
  }
  double acc[4] = {0, 0, 0, 0};
  for (int k = 0; k < nblocks; ++k)
    for (int c = 0; c < 4; ++c) acc[c] += partial[k * 4 + c];
  out[0] = acc[0] / acc[3];
  out[1] = acc[1] / acc[3];
  out[2] = acc[2] / acc[3];
  out[3] = acc[3];
}

// Bulk pressure of Eq. bulkp (e_2 = 1) at one node.
__global__ void bulk_pressure_kernel(ForceParams fp, const double *fields, int64_t s, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double cs2 = 1.0 / 3.0;
  const double nA = fields[s], nB = fields[fp.N + s], psA = fields[2 * fp.N + s], psB = fields[3 * fp.N + s];
  out[0] = (nA + nB) * cs2 + fp.G * cs2 * nA * nB + 0.5 * fp.G_self[0] * cs2 * psA * psA +
           0.5 * fp.G_self[1] * cs2 * psB * psB;
}

// sigma[R] minimum (section 3) on one warp; see sc_sigma_minimum in sc.h.
__global__ void __launch_bounds__(32) sigma_kernel(const double *rows, int nbins, const double *pio, int dim,
                                                   double R_lo, double R_hi, double R_step, double *out) {
  const int lane = threadIdx.x;
  __shared__ double s_C;
  if (lane == 0) {
    // trapezoid of r^(dim-1) P_T over the non-empty rows, in order
    double T = 0.0, rp = 0.0, fp = 0.0, rmax = 0.0;
    bool first = true;
    for (int b = 0; b < nbins; ++b) {
      if (rows[b * 6 + 5] <= 0.0) continue;
      const double r = rows[b * 6 + 0], pt = rows[b * 6 + 2];
      const double f = (dim == 3 ? r * r : r) * pt;
      if (!first) T += 0.5 * (f + fp) * (r - rp);
      first = false;
      rp = r;
      fp = f;
      rmax = r;
    }
    const double Pout = pio[1];
    s_C = Pout * (dim == 3 ? rmax * rmax * rmax / 3.0 : rmax * rmax / 2.0) - T;
  }
  __syncwarp();
  const double Pin = pio[0], Pout = pio[1], dP = Pin - Pout, C = s_C;
  auto sigma = [&](double R) { return dim == 3 ? dP * R / 3.0 + C / (R * R) : dP * R / 2.0 + C / R; };
  // grid search: each lane scans a strided subset, then a warp argmin (lowest index on ties)
  const int ng = int(floor((R_hi - R_lo) / R_step + 0.5)) + 1;
  double best = INFINITY;
  int bi = -1;
  for (int k = lane; k < ng; k += 32) {
    const double v = sigma(R_lo + k * R_step);
    if (v < best) {
      best = v;
      bi = k;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (oi >= 0 && (ob < best || (ob == best && (bi < 0 || oi < bi)))) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) {
    const double Rs = dim == 3 ? cbrt(6.0 * C / dP) : sqrt(2.0 * C / dP);
    out[0] = dP;
    out[1] = C;
    out[2] = Rs;
    out[3] = dim == 3 ? 0.5 * dP * Rs : dP * Rs;
    int k = bi < 1 ? 1 : (bi > ng - 2 ? ng - 2 : bi);
    double Rg = NAN, sg = NAN;
    if (ng >= 3) {
      const double y0 = sigma(R_lo + (k - 1) * R_step), y1 = sigma(R_lo + k * R_step),
                   y2 = sigma(R_lo + (k + 1) * R_step);
      const double den = y0 - 2.0 * y1 + y2;
      const double off = den != 0.0 ? 0.5 * (y0 - y2) / den : 0.0;
      Rg = R_lo + (k + off) * R_step;
      sg = y1 - 0.25 * (y0 - y2) * off;
    }
    out[4] = Rg;
    out[5] = sg;
    out[6] = Pin;
    out[7] = Pout;
  }
}

// Flat-interface tension (section 4): sigma_0 = sum over the planes z >= nbins / 2 of
// P_N(z) - P_T(z) from planar profile rows; one warp, lane-strided sums and a fixed
// shuffle tree (deterministic).
__global__ void __launch_bounds__(32) sigma0_kernel(const double *rows, int nbins, double *out) {
  const int lane = threadIdx.x;
  double acc = 0.0;
  for (int z = nbins / 2 + lane; z < nbins; z += 32) acc += rows[z * 6 + 1] - rows[z * 6 + 2];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) out[0] = acc;
}

// Curvature expansion of the surface tension (Eq. sigma_c),
// sigma_s = sigma_0 (1 - 2 delta x + c x^2), x = 1 / R_s, by least squares over n
// droplets: sigma_0 fitted (columns 1, x, x^2) or held at *sigma0 (columns x, x^2 on
// sigma_s / sigma_0 - 1); order 1 drops the x^2 column.  The normal equations are
// formed in x scaled by 1 / max|x| and solved by Gaussian elimination with partial
// pivoting; one thread, fixed order.  out = (sigma_0, delta, c (NaN for order 1), rms
// residual of sigma_s).
__global__ void curvature_fit_kernel(const double *Rs, const double *sig, int n, int order, const double *sigma0,
                                     double *out) {
  if (threadIdx.x != 0) return;
  const bool fixed = sigma0 != nullptr;
  const double s0f = fixed ? sigma0[0] : 0.0;
  double xm = 0.0;
  for (int i = 0; i < n; ++i) xm = fmax(xm, fabs(1.0 / Rs[i]));
  const double sc = xm > 0.0 ? 1.0 / xm : 1.0;
  const int m = fixed ? order : order + 1;
  double G[3][4];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 4; ++l) G[k][l] = 0.0;
  for (int i = 0; i < n; ++i) {
    const double t = sc / Rs[i];
    const double col[3] = {fixed ? t : 1.0, fixed ? t * t : t, t * t};
    const double y = fixed ? sig[i] / s0f - 1.0 : sig[i];
    for (int k = 0; k < m; ++k) {
      for (int l = 0; l < m; ++l) G[k][l] += col[k] * col[l];
      G[k][3] += col[k] * y;
    }
  }
  // elimination on the augmented m x (m + 1) system
  for (int k = 0; k < m; ++k) {
    int piv = k;
    for (int r = k + 1; r < m; ++r)
      if (fabs(G[r][k]) > fabs(G[piv][k])) piv = r;
    if (piv != k)
      for (int l = 0; l < 4; ++l) {
        const double t = G[k][l];
        G[k][l] = G[piv][l];
        G[piv][l] = t;
      }
    for (int r = k + 1; r < m; ++r) {
      const double f = G[r][k] / G[k][k];
      for (int l = k; l < 4; ++l) G[r][l] -= f * G[k][l];
    }
  }
  double c[3] = {0.0, 0.0, 0.0};
  for (int k = m - 1; k >= 0; --k) {
    double v = G[k][3];
    for (int l = k + 1; l < m; ++l) v -= G[k][l] * c[l];
    c[k] = v / G[k][k];
  }
  double s0, a1, a2;  // sigma_s = s0 + a1 x + a2 x^2 in unscaled x
  if (fixed) {
    s0 = s0f;
    a1 = s0f * c[0] * sc;
    a2 = order == 2 ? s0f * c[1] * sc * sc : 0.0;
  } else {
    s0 = c[0];
    a1 = c[1] * sc;
    a2 = order == 2 ? c[2] * sc * sc : 0.0;
  }
  double rss = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = 1.0 / Rs[i];
    const double d = s0 + a1 * x + a2 * x * x - sig[i];
    rss += d * d;
  }
  out[0] = s0;
  out[1] = -a1 / (2.0 * s0);
  out[2] = order == 2 ? a2 / s0 : NAN;
  out[3] = sqrt(rss / n);
}

// Deterministic FP64 totals: per-block partial sums (fixed grid-stride order,
// fixed tree) of mass_A, mass_B and momentum; finalised in block order.
template <int LAT, class ST>
__global__ void __launch_bounds__(256) totals_partial_kernel(PopArgs a, double *partial) {
  using L = Lattice<LAT>;
  const ST *buf = static_cast<const ST *>(a.buf);
  const int64_t N = a.N;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int J = 0; J < 2; ++J)
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        // stored at the collision site: sums over all sites need no pull
        const double f = pop_value<LAT, ST>(a, buf, i, J, s);
        acc[J] += f;
#pragma unroll
        for (int m = 0; m < 3; ++m) acc[2 + m] += L::c(i, m) * f;
      }
  }
  __shared__ double red[5][256];
#pragma unroll
  for (int c = 0; c < 5; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int c = 0; c < 5; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void totals_finalize_kernel(const double *partial, int nblocks, int ncomp, double *out) {
  const int c = threadIdx.x;
  if (c >= ncomp) return;
  double acc = 0.0;
  for (int k = 0; k < nblocks; ++k) acc += partial[k * ncomp + c];
  out[c] = acc;
}

// Deterministic FP64 sums of two fields (used for the mean initial densities).
__global__ void __launch_bounds__(256) sum2_partial_kernel(const double *a, const double *b, int64_t N,
                                                           double *partial) {
  double acc[2] = {0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    acc[0] += a[s];
    acc[1] += b[s];
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = acc[0];
  red[1][threadIdx.x] = acc[1];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) partial[blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x][0];
}

// max |n_J - nbar_J| of both init fields (for the F16/BF16 scales); one value per block.
__global__ void __launch_bounds__(256) maxdev_partial_kernel(const double *a, const double *b, int64_t N,
                                                             double nbarA, double nbarB, double *partial) {
  double m[2] = {0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    m[0] = fmax(m[0], fabs(a[s] - nbarA));
    m[1] = fmax(m[1], fabs(b[s] - nbarB));
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = m[0];
  red[1][threadIdx.x] = m[1];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + w]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) partial[blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x][0];
}

// min of (n_A, n_B) over both init fields, per block (validation: densities > 0).
__global__ void __launch_bounds__(256) min2_partial_kernel(const double *a, const double *b, int64_t N,
                                                           double *partial) {
  double m = INFINITY;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x)
    m = fmin(m, fmin(a[s], b[s]));  // NaN-propagation: fmin ignores NaN, so flag it explicitly
  __shared__ double red[256];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x)
    if (!(a[s] > 0.0) || !(b[s] > 0.0) || !isfinite(a[s]) || !isfinite(b[s])) bad = 1;
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = bad ? -1.0 : red[0];
}

}  // namespace scgb
