// sc_pressure_profile_noalloc: the pressure-tensor profile for callers that
// cannot allocate device memory.  Its only scratch (per-block partial sums) is
// a fixed file-scope __device__ array of this library, so the call allocates
// nothing; the caller passes the density fields and the output rows.  The
// profile kernels are the ones sc_pressure_profile launches (sc_profile.cuh),
// reading psi from the densities on the fly instead of from stored planes.
#include <mutex>

#include "sc_host.h"

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

// Device address of the scratch array on the current device.  In host code the
// name g_profile_scratch is a host-side stand-in, not a device address, so the
// address is asked of the runtime, with the device current.  It is asked again
// on every call whose stream is not capturing (a device reset reloads the module
// and may move the array); a call made while the stream captures a graph takes
// the address an earlier call on this device found, and fails if there is none.
sc_status scratch_on_current_device(cudaStream_t stream, double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(SC_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(SC_EUNSUPPORTED, "device index beyond the scratch table");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return set_error(SC_ECUDA, cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_profile_scratch);
    if (e != cudaSuccess) return set_error(SC_ECUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double *>(p);
  } else if (!g_scratch_ptr[dev]) {
    return set_error(SC_EINVAL, "the first sc_pressure_profile_noalloc call on a device must come before any "
                                "stream capture (it looks up the scratch array's device address)");
  }
  *out = g_scratch_ptr[dev];
  return SC_OK;
}

}  // namespace

extern "C" sc_status sc_pressure_profile_noalloc(const sc_params *p, const double *nA, const double *nB, int32_t kind,
                                                 const double centre[3], double bin_width, int32_t nbins, double *out,
                                                 void *stream) {
  if (!p || !nA || !nB || !centre || !out) return set_error(SC_EINVAL, "params, nA, nB, centre and out must be non-NULL");
  // the same model checks sc_create applies, so both profile entry points accept the same parameters
  sc_status st = validate_model(p);
  if (st != SC_OK) return st;
  if (nbins > kMaxBins)
    return set_error(SC_EINVAL, "nbins must be in [1, 4096] (the fixed scratch of sc_pressure_profile_noalloc)");
  st = validate_profile_request(p, kind, centre, bin_width, nbins, kMaxBins);
  if (st != SC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *scratch = nullptr;
  st = scratch_on_current_device(s, &scratch);
  if (st != SC_OK) return st;
  ForceParams fp;
  fp.G = p->G;
  fp.G_self[0] = p->G_self[0];
  fp.G_self[1] = p->G_self[1];
  fp.nx = p->nx;
  fp.ny = p->ny;
  fp.nz = p->nz;
  fp.N = (int64_t)p->nx * p->ny * p->nz;
  // as many blocks as the scratch holds rows for (at most kMaxBlocks, at least one)
  const cudaError_t e = launch_profile(p->lattice, p->stencil, fp, profile_args(p, kind, centre, bin_width, nbins),
                                       DensityFields{nA, nB, p->psi_self == SC_PSI_EXP ? 1 : 0}, scratch,
                                       kScratchDoubles, kMaxBlocks, out, s);
  if (e != cudaSuccess) return set_error(SC_ECUDA, cudaGetErrorString(e));
  return SC_OK;
}
