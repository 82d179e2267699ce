// The lattice pressure tensor of Eq. sm:pt in FP64 and its profiles (section 3,
// Eq. pt_projection: radial shells; section 4: planes of a flat interface; the
// paper's own x-axis line).  One implementation serves both profile entry points:
// the kernels are templated on where the fields come from -- the [4][N] FP64
// planes (n_A, n_B, psi_A, psi_B) a context computes from its state, or bare
// density fields with the pseudopotential evaluated on the fly.
#pragma once

#include "sc_common.cuh"

namespace scgb {

__device__ __forceinline__ void coords(int64_t s, int nx, int ny, int &x, int &y, int &z) {
  x = int(s % nx);
  const int64_t r = s / nx;
  y = int(r % ny);
  z = int(r / ny);
}
__device__ __forceinline__ int64_t site_at(int x, int y, int z, int nx, int ny, int nz) {
  x = ((x % nx) + nx) % nx;
  y = ((y % ny) + ny) % ny;
  z = ((z % nz) + nz) % nz;
  return (int64_t)x + (int64_t)nx * (y + (int64_t)ny * z);
}

struct ForceParams {
  double G, G_self[2];
  int nx, ny, nz;
  int64_t N;
};

// Field f of {n_A, n_B, psi_A, psi_B} at site s from stored FP64 planes [4][N].
struct StoredFields {
  const double *f;
  int64_t N;
  __device__ __forceinline__ double operator()(int k, int64_t s) const { return f[k * N + s]; }
};

// The same four fields from two density arrays; psi = exp(-1/n) or psi = n
// (section 4), evaluated where it is needed.
struct DensityFields {
  const double *nA, *nB;
  int psi_exp;
  __device__ __forceinline__ double operator()(int k, int64_t s) const {
    const double n = (k & 1) ? nB[s] : nA[s];
    return (k < 2 || !psi_exp) ? n : exp(-1.0 / n);
  }
};

// Lattice pressure tensor of Eq. sm:pt at one site; P = {xx, yy, zz, xy, xz, yz}.
template <int LAT, int STEN, class FA>
__device__ __forceinline__ void ptensor64(const ForceParams &p, const FA &fld, int x, int y, int z, int64_t s,
                                          double P[6]) {
  using SN = Stencil<LAT, STEN>;
  const double cs2 = 1.0 / 3.0;
  constexpr int MU[6] = {0, 1, 2, 0, 0, 1}, NU[6] = {0, 1, 2, 1, 2, 2};
  double C[4][6];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int c = 0; c < 6; ++c) C[f][c] = 0.0;
#pragma unroll
  for (int k = 0; k < SN::NH; ++k) {
    const int v[3] = {SN::v(k, 0), SN::v(k, 1), SN::v(k, 2)};
    const int64_t sp = site_at(x + v[0], y + v[1], z + v[2], p.nx, p.ny, p.nz);
    const int64_t sm = site_at(x - v[0], y - v[1], z - v[2], p.nx, p.ny, p.nz);
    const double W = SN::W(k);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const double sum = fld(f, sp) + fld(f, sm);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const int vv = v[MU[c]] * v[NU[c]];
        if (vv) C[f][c] += W * vv * sum;
      }
    }
  }
  const double nA = fld(0, s), nB = fld(1, s), psA = fld(2, s), psB = fld(3, s);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const double ideal = c < 3 ? (nA + nB) * cs2 : 0.0;
    P[c] = ideal + 0.5 * p.G * cs2 * nA * C[1][c] + 0.5 * p.G * cs2 * nB * C[0][c] +
           0.5 * p.G_self[0] * cs2 * psA * C[2][c] + 0.5 * p.G_self[1] * cs2 * psB * C[3][c];
  }
}

struct ProfileArgs {
  int kind;  // sc_profile_kind
  double centre[3];
  double bin_width;
  int nbins;
  int dim;   // 2 or 3
  int64_t chunk;  // sites per block
};

// Per-block partial sums of a profile: one warp per block accumulates into its
// own shared-memory bins, lane by lane in a fixed order (deterministic), then
// writes rows [nbins][6] = (sum coordinate, sum P_N, sum P_T, sum n_A, sum n_B, count).
// Every row of the block's slice of `partial` is written, so nothing left there
// by an earlier launch is ever read.
template <int LAT, int STEN, class FA>
__global__ void __launch_bounds__(32) profile_partial_kernel(ForceParams fp, ProfileArgs pa, FA fld,
                                                             double *partial) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *bins = reinterpret_cast<double *>(smem_raw);
  const int lane = threadIdx.x;
  for (int k = lane; k < pa.nbins * 6; k += 32) bins[k] = 0.0;
  __syncwarp();
  const int64_t N = fp.N;
  const int64_t s0 = blockIdx.x * pa.chunk, s1 = min(N, s0 + pa.chunk);
  const int cx = int(floor(pa.centre[0] + 0.5)), cy = int(floor(pa.centre[1] + 0.5)),
            cz = int(floor(pa.centre[2] + 0.5));
  for (int64_t base = s0; base < s1; base += 32) {
    const int64_t s = base + lane;
    int bin = -1;
    double vals[5] = {0, 0, 0, 0, 0};
    if (s < s1) {
      int x, y, z;
      coords(s, fp.nx, fp.ny, x, y, z);
      double coord = 0.0, d[3] = {0, 0, 0};
      if (pa.kind == SC_PROFILE_RADIAL) {
        const int c[3] = {x, y, z}, L[3] = {fp.nx, fp.ny, fp.nz};
        double r2 = 0.0;
        for (int m = 0; m < 3; ++m) {
          double dd = c[m] - pa.centre[m];
          dd -= L[m] * floor(dd / L[m] + 0.5);  // minimum image
          d[m] = dd;
          r2 += dd * dd;
        }
        coord = sqrt(r2);
        bin = int(floor(coord / pa.bin_width));
      } else if (pa.kind == SC_PROFILE_PLANAR_Z) {
        coord = z;
        bin = z;
      } else {
        // the x axis through the centre node: row k is the site (cx + k, cy, cz); the
        // entry points accept nbins <= nx only, so each row holds exactly one site
        const int k = ((x - cx) % fp.nx + fp.nx) % fp.nx;
        if (y == ((cy % fp.ny) + fp.ny) % fp.ny && z == ((cz % fp.nz) + fp.nz) % fp.nz) {
          coord = k;
          bin = k;
        }
      }
      if (bin >= pa.nbins) bin = -1;
      if (bin >= 0) {
        double P[6];
        ptensor64<LAT, STEN>(fp, fld, x, y, z, s, P);
        double PN, PT;
        if (pa.kind == SC_PROFILE_RADIAL) {
          const double tr = pa.dim == 3 ? P[0] + P[1] + P[2] : P[0] + P[1];
          if (coord == 0.0) {
            PN = PT = tr / pa.dim;
          } else {
            const double e[3] = {d[0] / coord, d[1] / coord, d[2] / coord};
            PN = e[0] * e[0] * P[0] + e[1] * e[1] * P[1] + e[2] * e[2] * P[2] + 2.0 * e[0] * e[1] * P[3] +
                 2.0 * e[0] * e[2] * P[4] + 2.0 * e[1] * e[2] * P[5];
            PT = (tr - PN) / (pa.dim - 1);
          }
        } else if (pa.kind == SC_PROFILE_PLANAR_Z) {
          PN = P[2];
          PT = 0.5 * (P[0] + P[1]);
        } else {
          PN = P[0];
          PT = P[1];
        }
        vals[0] = coord;
        vals[1] = PN;
        vals[2] = PT;
        vals[3] = fld(0, s);
        vals[4] = fld(1, s);
      }
    }
    // fixed-order accumulation: lane l's contribution is added in iteration l
    for (int l = 0; l < 32; ++l) {
      const int b = __shfl_sync(0xffffffffu, bin, l);
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const double t = __shfl_sync(0xffffffffu, vals[c], l);
        if (lane == c) v = t;
      }
      if (b >= 0 && lane < 6) bins[b * 6 + lane] += (lane == 5) ? 1.0 : v;
      __syncwarp();
    }
  }
  __syncwarp();
  double *out = partial + (int64_t)blockIdx.x * pa.nbins * 6;
  for (int k = lane; k < pa.nbins * 6; k += 32) out[k] = bins[k];
}

// Sum the per-block partials in block order and turn sums into means.
template <class T>
__global__ void profile_finalize_kernel(const T *partial, int nblocks, int nbins, T *out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
    T acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < nblocks; ++k)
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[c] += partial[((int64_t)k * nbins + b) * 6 + c];
    const T cnt = acc[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) out[b * 6 + c] = cnt > 0 ? acc[c] / cnt : T(0);
    out[b * 6 + 5] = cnt;
  }
}

// Blocks of a profile launch and the sites each one takes (a multiple of 32):
// as many blocks as `partial_doubles` holds rows for, at most max_blocks and at
// most one per 32 sites.
inline int64_t profile_blocks(int64_t N, int nbins, int64_t partial_doubles, int64_t max_blocks, int64_t *chunk) {
  int64_t blocks = partial_doubles / ((int64_t)nbins * 6);
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks > (N + 31) / 32) blocks = (N + 31) / 32;
  if (blocks < 1) blocks = 1;
  int64_t c = (N + blocks - 1) / blocks;
  c = (c + 31) / 32 * 32;
  *chunk = c;
  return (N + c - 1) / c;
}

// Launch the partial and finalise kernels of one profile on stream st.
template <int LAT, int STEN, class FA>
cudaError_t launch_profile_lat(const ForceParams &fp, ProfileArgs pa, const FA &fld, double *partial,
                               int64_t partial_doubles, int64_t max_blocks, double *out, cudaStream_t st) {
  const int64_t blocks = profile_blocks(fp.N, pa.nbins, partial_doubles, max_blocks, &pa.chunk);
  const size_t row_bytes = (size_t)pa.nbins * 6 * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(profile_partial_kernel<LAT, STEN, FA>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_bytes);
  if (e != cudaSuccess) return e;
  profile_partial_kernel<LAT, STEN, FA><<<(int)blocks, 32, row_bytes, st>>>(fp, pa, fld, partial);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  profile_finalize_kernel<double><<<(pa.nbins + 127) / 128, 128, 0, st>>>(partial, (int)blocks, pa.nbins, out);
  return cudaGetLastError();
}

// Dispatch on the lattice and stencil (D2Q9 takes E4 only).
template <class FA>
cudaError_t launch_profile(int lattice, int stencil, const ForceParams &fp, const ProfileArgs &pa, const FA &fld,
                           double *partial, int64_t partial_doubles, int64_t max_blocks, double *out,
                           cudaStream_t st) {
  if (lattice == SC_D2Q9) return launch_profile_lat<kD2Q9, kE4>(fp, pa, fld, partial, partial_doubles, max_blocks, out, st);
  if (stencil == SC_FORCE_E6)
    return launch_profile_lat<kD3Q19, kE6>(fp, pa, fld, partial, partial_doubles, max_blocks, out, st);
  return launch_profile_lat<kD3Q19, kE4>(fp, pa, fld, partial, partial_doubles, max_blocks, out, st);
}

}  // namespace scgb
