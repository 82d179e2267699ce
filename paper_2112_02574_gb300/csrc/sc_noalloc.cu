// sc_pressure_profile_noalloc: the pressure-tensor profile for callers that
// cannot allocate device memory.  Its only scratch (per-block partial sums) is
// a fixed file-scope __device__ array of this library, so the call allocates
// nothing; the caller passes the density fields and the output rows.
#include <mutex>

#include "sc_common.cuh"

namespace scgb {
sc_status set_error(sc_status st, const char *msg);  // sc_api.cu: records sc_last_error()
}

using namespace scgb;

namespace {

// Scratch: per-block partial rows [blocks][nbins][6], FP64.  4 MiB, held by every
// GPU that loads this library until the process exits.
constexpr int64_t kScratchDoubles = int64_t(1) << 19;
constexpr int kMaxBins = 4096;   // shared-memory bins of one block (nbins x 48 B)
constexpr int kMaxBlocks = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_profile_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per
// device, with that device current).  The name g_profile_scratch is a host-side
// stand-in in host code, not a device address.
sc_status scratch_on_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(SC_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(SC_EUNSUPPORTED, "device index beyond the scratch table");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_profile_scratch);
    if (e != cudaSuccess) return set_error(SC_ECUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return SC_OK;
}

struct NoallocArgs {
  const double *nA, *nB;
  int nx, ny, nz;
  int64_t N;
  double G, G_self[2];
  int psi_exp;
  int kind;
  double centre[3];
  double bin_width;
  int nbins;
  int dim;
  int64_t chunk;
};

__device__ __forceinline__ int64_t wrap_site(int x, int y, int z, int nx, int ny, int nz) {
  x = ((x % nx) + nx) % nx;
  y = ((y % ny) + ny) % ny;
  z = ((z % nz) + nz) % nz;
  return (int64_t)x + (int64_t)nx * (y + (int64_t)ny * z);
}

__device__ __forceinline__ double psi_of(const NoallocArgs &a, double n) { return a.psi_exp ? exp(-1.0 / n) : n; }

// Eq. sm:pt at one site from the density fields, psi evaluated on the fly.
template <int LAT, int STEN>
__device__ void tensor_at(const NoallocArgs &a, int x, int y, int z, int64_t s, double P[6]) {
  using SN = Stencil<LAT, STEN>;
  const double cs2 = 1.0 / 3.0;
  constexpr int MU[6] = {0, 1, 2, 0, 0, 1}, NU[6] = {0, 1, 2, 1, 2, 2};
  double C[4][6];
  for (int f = 0; f < 4; ++f)
    for (int c = 0; c < 6; ++c) C[f][c] = 0.0;
#pragma unroll
  for (int k = 0; k < SN::NH; ++k) {
    const int v[3] = {SN::v(k, 0), SN::v(k, 1), SN::v(k, 2)};
    const int64_t sp = wrap_site(x + v[0], y + v[1], z + v[2], a.nx, a.ny, a.nz);
    const int64_t sm = wrap_site(x - v[0], y - v[1], z - v[2], a.nx, a.ny, a.nz);
    const double W = SN::W(k);
    const double nAp = a.nA[sp], nAm = a.nA[sm], nBp = a.nB[sp], nBm = a.nB[sm];
    const double sum[4] = {nAp + nAm, nBp + nBm, psi_of(a, nAp) + psi_of(a, nAm), psi_of(a, nBp) + psi_of(a, nBm)};
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const int vv = v[MU[c]] * v[NU[c]];
        if (vv) C[f][c] += W * vv * sum[f];
      }
  }
  const double nA = a.nA[s], nB = a.nB[s], psA = psi_of(a, nA), psB = psi_of(a, nB);
  for (int c = 0; c < 6; ++c) {
    const double ideal = c < 3 ? (nA + nB) * cs2 : 0.0;
    P[c] = ideal + 0.5 * a.G * cs2 * nA * C[1][c] + 0.5 * a.G * cs2 * nB * C[0][c] +
           0.5 * a.G_self[0] * cs2 * psA * C[2][c] + 0.5 * a.G_self[1] * cs2 * psB * C[3][c];
  }
}

// Per-block partial rows, one warp per block accumulating lane by lane (fixed order).
template <int LAT, int STEN>
__global__ void __launch_bounds__(32) noalloc_partial_kernel(NoallocArgs a, double *partial) {
  extern __shared__ __align__(16) unsigned char smem_bins[];
  double *bins = reinterpret_cast<double *>(smem_bins);
  const int lane = threadIdx.x;
  for (int k = lane; k < a.nbins * 6; k += 32) bins[k] = 0.0;
  __syncwarp();
  const int64_t s0 = blockIdx.x * a.chunk, s1 = min(a.N, s0 + a.chunk);
  const int cx = int(floor(a.centre[0] + 0.5)), cy = int(floor(a.centre[1] + 0.5)), cz = int(floor(a.centre[2] + 0.5));
  for (int64_t base = s0; base < s1; base += 32) {
    const int64_t s = base + lane;
    int bin = -1;
    double vals[5] = {0, 0, 0, 0, 0};
    if (s < s1) {
      const int x = int(s % a.nx), y = int((s / a.nx) % a.ny), z = int(s / ((int64_t)a.nx * a.ny));
      double coord = 0.0, d[3] = {0, 0, 0};
      if (a.kind == SC_PROFILE_RADIAL) {
        const int c[3] = {x, y, z}, L[3] = {a.nx, a.ny, a.nz};
        double r2 = 0.0;
        for (int m = 0; m < 3; ++m) {
          double dd = c[m] - a.centre[m];
          dd -= L[m] * floor(dd / L[m] + 0.5);
          d[m] = dd;
          r2 += dd * dd;
        }
        coord = sqrt(r2);
        bin = int(floor(coord / a.bin_width));
      } else if (a.kind == SC_PROFILE_PLANAR_Z) {
        coord = z;
        bin = z;
      } else {
        const int k = ((x - cx) % a.nx + a.nx) % a.nx;
        if (y == ((cy % a.ny) + a.ny) % a.ny && z == ((cz % a.nz) + a.nz) % a.nz) {
          coord = k;
          bin = k;
        }
      }
      if (bin >= a.nbins) bin = -1;
      if (bin >= 0) {
        double P[6];
        tensor_at<LAT, STEN>(a, x, y, z, s, P);
        double PN, PT;
        if (a.kind == SC_PROFILE_RADIAL) {
          const double tr = a.dim == 3 ? P[0] + P[1] + P[2] : P[0] + P[1];
          if (coord == 0.0) {
            PN = PT = tr / a.dim;
          } else {
            const double e[3] = {d[0] / coord, d[1] / coord, d[2] / coord};
            PN = e[0] * e[0] * P[0] + e[1] * e[1] * P[1] + e[2] * e[2] * P[2] + 2.0 * e[0] * e[1] * P[3] +
                 2.0 * e[0] * e[2] * P[4] + 2.0 * e[1] * e[2] * P[5];
            PT = (tr - PN) / (a.dim - 1);
          }
        } else if (a.kind == SC_PROFILE_PLANAR_Z) {
          PN = P[2];
          PT = 0.5 * (P[0] + P[1]);
        } else {
          PN = P[0];
          PT = P[1];
        }
        vals[0] = coord;
        vals[1] = PN;
        vals[2] = PT;
        vals[3] = a.nA[s];
        vals[4] = a.nB[s];
      }
    }
    for (int l = 0; l < 32; ++l) {
      const int b = __shfl_sync(0xffffffffu, bin, l);
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const double t = __shfl_sync(0xffffffffu, vals[c], l);
        if (lane == c) v = t;
      }
      if (b >= 0 && lane < 6) bins[b * 6 + lane] += (lane == 5) ? 1.0 : v;
    }
  }
  __syncwarp();
  // every entry this call's finalise step reads is written here: nothing left
  // in the scratch array by an earlier call is ever read
  double *out = partial + (int64_t)blockIdx.x * a.nbins * 6;
  for (int k = lane; k < a.nbins * 6; k += 32) out[k] = bins[k];
}

__global__ void noalloc_finalize_kernel(const double *partial, int nblocks, int nbins, double *out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < nblocks; ++k)
      for (int c = 0; c < 6; ++c) acc[c] += partial[((int64_t)k * nbins + b) * 6 + c];
    const double cnt = acc[5];
    for (int c = 0; c < 5; ++c) out[b * 6 + c] = cnt > 0 ? acc[c] / cnt : 0.0;
    out[b * 6 + 5] = cnt;
  }
}

template <int LAT, int STEN>
cudaError_t launch_partial(const NoallocArgs &a, int blocks, double *partial, cudaStream_t s) {
  const size_t smem = (size_t)a.nbins * 6 * sizeof(double);
  cudaError_t e =
      cudaFuncSetAttribute(noalloc_partial_kernel<LAT, STEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  noalloc_partial_kernel<LAT, STEN><<<blocks, 32, smem, s>>>(a, partial);
  return cudaGetLastError();
}

}  // namespace

extern "C" sc_status sc_pressure_profile_noalloc(const sc_params *p, const double *nA, const double *nB, int32_t kind,
                                                 const double centre[3], double bin_width, int32_t nbins, double *out,
                                                 void *stream) {
  if (!p || !nA || !nB || !centre || !out) return set_error(SC_EINVAL, "params, nA, nB, centre and out must be non-NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return set_error(SC_EINVAL, "lattice size must be >= 1");
  if (p->lattice != SC_D2Q9 && p->lattice != SC_D3Q19) return set_error(SC_EINVAL, "unknown lattice");
  if (p->lattice == SC_D2Q9 && (p->nz != 1 || p->stencil != SC_FORCE_E4))
    return set_error(SC_EINVAL, "D2Q9 needs nz == 1 and the E4 stencil");
  if (p->stencil != SC_FORCE_E4 && p->stencil != SC_FORCE_E6) return set_error(SC_EINVAL, "unknown stencil");
  if (kind < SC_PROFILE_RADIAL || kind > SC_PROFILE_AXIS_X) return set_error(SC_EINVAL, "unknown profile kind");
  if (kind == SC_PROFILE_RADIAL && !(bin_width > 0.0)) return set_error(SC_EINVAL, "bin_width must be > 0");
  if (nbins < 1 || nbins > kMaxBins)
    return set_error(SC_EINVAL, "nbins must be in [1, 4096] (the fixed scratch of sc_pressure_profile_noalloc)");
  for (int m = 0; m < 3; ++m)
    if (!isfinite(centre[m])) return set_error(SC_EINVAL, "centre must be finite");
  double *scratch = nullptr;
  sc_status st = scratch_on_current_device(&scratch);
  if (st != SC_OK) return st;
  NoallocArgs a;
  a.nA = nA;
  a.nB = nB;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.N = (int64_t)p->nx * p->ny * p->nz;
  a.G = p->G;
  a.G_self[0] = p->G_self[0];
  a.G_self[1] = p->G_self[1];
  a.psi_exp = p->psi_self == SC_PSI_EXP ? 1 : 0;
  a.kind = kind;
  for (int m = 0; m < 3; ++m) a.centre[m] = centre[m];
  a.bin_width = bin_width;
  a.nbins = nbins;
  a.dim = (p->lattice == SC_D3Q19 && p->nz > 1) ? 3 : 2;
  // as many blocks as the scratch holds rows for (at most kMaxBlocks, at least one)
  int64_t blocks = kScratchDoubles / ((int64_t)nbins * 6);
  if (blocks > kMaxBlocks) blocks = kMaxBlocks;
  if (blocks > (a.N + 31) / 32) blocks = (a.N + 31) / 32;
  if (blocks < 1) blocks = 1;
  a.chunk = (a.N + blocks - 1) / blocks;
  a.chunk = (a.chunk + 31) / 32 * 32;
  blocks = (a.N + a.chunk - 1) / a.chunk;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (p->lattice == SC_D2Q9)
    e = launch_partial<kD2Q9, kE4>(a, (int)blocks, scratch, s);
  else if (p->stencil == SC_FORCE_E6)
    e = launch_partial<kD3Q19, kE6>(a, (int)blocks, scratch, s);
  else
    e = launch_partial<kD3Q19, kE4>(a, (int)blocks, scratch, s);
  if (e == cudaSuccess) {
    noalloc_finalize_kernel<<<(nbins + 127) / 128, 128, 0, s>>>(scratch, (int)blocks, nbins, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_error(SC_ECUDA, cudaGetErrorString(e));
  return SC_OK;
}
