// C ABI of the library (declared in include/sc.h): validation, workspace
// layout, contexts, and the host side of every entry point.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>

#include "sc_aux.cuh"
#include "sc_dispatch.h"
#include "sc_host.h"

using namespace scgb;

namespace {

thread_local std::string g_err;

sc_status fail(sc_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define SC_CUDA(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(SC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

constexpr size_t kAlign = 256;
constexpr size_t kPartialBytes = size_t(16) << 20;  // per-block partial sums of the reductions
constexpr size_t kStatusBytes = 4096;                // status word + small scalars
constexpr int kMaxProfileBins = 4096;
// rows of a profile kept for sc_surface_of_tension ([kMaxProfileBins][6] FP64), then P_in, P_out
constexpr size_t kAnalysisBytes = (size_t)kMaxProfileBins * 6 * sizeof(double) + 256;
constexpr int kMaxPartialBlocks = 1024;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int q_of(const sc_params *p) { return p->lattice == SC_D3Q19 ? 19 : 9; }
size_t store_bytes(int storage) {
  switch (storage) {
    case SC_STORE_F32: return 4;
    case SC_STORE_F16:
    case SC_STORE_BF16: return 2;
    case SC_STORE_F64: return 8;
    default: return 0;
  }
}

// Sites per 16-byte copy chunk of a population row (both components).
int chunk_sites(int storage) { return storage == SC_STORE_F64 ? 1 : (storage == SC_STORE_F32 ? 2 : 4); }

bool staged_eligible(const sc_params *p, int tile_y) {
  if (p->lattice != SC_D3Q19 || p->stencil != SC_FORCE_E4 || p->nx < 32 || p->nx % chunk_sites(p->storage) != 0)
    return false;
  if (p->storage == SC_STORE_F64) return tile_y == 4;
  return tile_y == 4 || tile_y == 8 || tile_y == 16;
}

// Kernel choice and tiles (measured sweeps at 128^3, 256^3 and 512^3 set the defaults).
bool is_16bit(int storage) { return storage == SC_STORE_F16 || storage == SC_STORE_BF16; }
// tau_A = tau_B = 1: the step kernels' instantiation that carries momentum sums instead of populations.
bool tau_one(const sc_params *p) { return p->tau[0] == 1.0 && p->tau[1] == 1.0; }
// Tile 32 x 8 for 16-bit storage, and for FP32 with tau = 1, whose momentum carry leaves room for three
// 8-warp blocks per SM (80 registers, no spills; same box at 128^3: FP32 126.3 -> 120.0 us against tile
// 32 x 4 with four blocks, FP16 101.5 -> 98.0 us against two blocks per SM); FP64 and FP32 with tau != 1
// keep tile 32 x 4 (their populations carried across the plane delay need the registers).
int staged_default_tile_y(const sc_params *p) {
  if (is_16bit(p->storage)) return 8;
  return (p->storage == SC_STORE_F32 && tau_one(p)) ? 8 : 4;
}
bool use_staged(const sc_params *p) {
  if (p->variant == 1) return false;
  return staged_eligible(p, p->tile_y ? p->tile_y : staged_default_tile_y(p));
}
int default_tile_y(const sc_params *p) {
  if (p->tile_y) return p->tile_y;
  if (use_staged(p)) return staged_default_tile_y(p);
  return p->lattice == SC_D3Q19 ? 8 : 4;
}
// F32 tile 32 x 4: one stage and three resident blocks per SM beat two stages and two
// blocks, with and without a self coupling (128^3 .. 512^3, same-box comparisons);
// F64 keeps two stages (three of its blocks do not fit in registers).
bool has_self(const sc_params *p) { return p->G_self[0] != 0.0 || p->G_self[1] != 0.0; }

int effective_stages(const sc_params *p, int tile_y) {
  if (p->stages) return p->stages;
  if (tile_y == 4) return p->storage == SC_STORE_F64 ? 2 : 1;
  return 1;
}
int effective_blocks_per_sm(const sc_params *p, int tile_y) {
  if (p->blocks_per_sm) return p->blocks_per_sm;
  if (tile_y == 4) return p->storage == SC_STORE_F64 ? 2 : 3;
  if (tile_y == 8) return (tau_one(p) && effective_stages(p, tile_y) == 1) ? 3 : 2;
  return 1;
}
int default_tile_z(const sc_params *p) {
  if (p->lattice == SC_D2Q9) return 1;
  const int want = p->tile_z ? p->tile_z : 32;
  return want < p->nz ? want : p->nz;
}

sc_status validate(const sc_params *p) {
  sc_status st = validate_model(p);
  if (st != SC_OK) return st;
  if (store_bytes(p->storage) == 0) return fail(SC_EINVAL, "unknown storage %d", p->storage);
  if (p->tile_y != 0 && p->tile_y != 1 && p->tile_y != 2 && p->tile_y != 4 && p->tile_y != 8 && p->tile_y != 16)
    return fail(SC_EINVAL, "tile_y must be 0, 1, 2, 4, 8 or 16");
  if (p->tile_z < 0) return fail(SC_EINVAL, "tile_z must be >= 0");
  if (p->variant < 0 || p->variant > 2) return fail(SC_EINVAL, "variant must be 0, 1 or 2");
  if (p->stages < 0 || p->stages > 2) return fail(SC_EINVAL, "stages must be 0, 1 or 2");
  if (p->blocks_per_sm < 0 || p->blocks_per_sm > 3) return fail(SC_EINVAL, "blocks_per_sm must be 0 .. 3");
  if (p->variant == 2 && !staged_eligible(p, p->tile_y ? p->tile_y : staged_default_tile_y(p)))
    return fail(SC_EINVAL, "the staged step kernel needs D3Q19, E4, nx >= 32, nx a multiple of %d for this "
                           "storage and tile_y 4, 8 or 16 (4 for F64 storage)", chunk_sites(p->storage));
  if (p->tile_y == 16 && !use_staged(p)) return fail(SC_EINVAL, "tile_y 16 needs the staged kernel");
  if (use_staged(p)) {
    const int ty = default_tile_y(p);
    const int lo = ty == 4 ? 2 : 1, hi = ty == 4 ? 3 : (ty == 8 ? (effective_stages(p, ty) == 1 ? 3 : 2) : 1);
    if (p->blocks_per_sm && (p->blocks_per_sm < lo || p->blocks_per_sm > hi))
      return fail(SC_EINVAL, "blocks_per_sm must be 0 or %d .. %d for the staged kernel with tile_y %d", lo, hi, ty);
    if (ty == 16 && effective_stages(p, ty) == 2 && !is_16bit(p->storage))
      return fail(SC_EINVAL, "two stages of 32 x 16 tiles exceed shared memory in this storage");
  }
  for (int J = 0; J < 2; ++J)
    if (!(p->tau[J] > 0.5) || !isfinite(p->tau[J])) return fail(SC_EINVAL, "tau[%d] must be > 1/2", J);
  return SC_OK;
}

struct Layout {
  size_t pop_bytes;  // one population buffer
  size_t ref_bytes;  // one local-reference density buffer (16-bit storage), else 0
  size_t off_pop[2], off_ref[2], off_fields, off_partial, off_status, off_analysis, total;
};

bool is_local_ref(int storage) { return storage == SC_STORE_F16 || storage == SC_STORE_BF16; }

Layout layout_of(const sc_params *p) {
  Layout L;
  const int64_t N = (int64_t)p->nx * p->ny * p->nz;
  L.pop_bytes = (size_t)2 * q_of(p) * N * store_bytes(p->storage);
  size_t off = 0;
  L.off_pop[0] = off;
  off = align_up(off + L.pop_bytes);
  L.off_pop[1] = off;
  off = align_up(off + L.pop_bytes);
  L.ref_bytes = is_local_ref(p->storage) ? (size_t)N * 2 * sizeof(float) : 0;
  L.off_ref[0] = off;
  off = align_up(off + L.ref_bytes);
  L.off_ref[1] = off;
  off = align_up(off + L.ref_bytes);
  L.off_fields = off;
  off = align_up(off + (size_t)4 * N * sizeof(double));
  L.off_partial = off;
  off = align_up(off + kPartialBytes);
  L.off_status = off;
  off = align_up(off + kStatusBytes);
  L.off_analysis = off;
  off = align_up(off + kAnalysisBytes);
  L.total = off;
  return L;
}


}  // namespace

// Records the calling thread's sc_last_error() message for entry points defined
// in other translation units of the library.
sc_status scgb::set_error(sc_status st, const char *msg) { return fail(st, "%s", msg); }

sc_status scgb::validate_model(const sc_params *p) {
  if (!p) return fail(SC_EINVAL, "params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(SC_EINVAL, "lattice size must be >= 1 in every direction");
  if ((int64_t)p->nx * p->ny * p->nz > (int64_t(1) << 31) - 1)
    return fail(SC_EINVAL, "more than 2^31 - 1 sites is not supported");
  if (p->lattice != SC_D2Q9 && p->lattice != SC_D3Q19) return fail(SC_EINVAL, "unknown lattice %d", p->lattice);
  if (p->lattice == SC_D2Q9 && p->nz != 1) return fail(SC_EINVAL, "D2Q9 needs nz == 1");
  if (p->stencil != SC_FORCE_E4 && p->stencil != SC_FORCE_E6) return fail(SC_EINVAL, "unknown stencil %d", p->stencil);
  if (p->stencil == SC_FORCE_E6 && p->lattice != SC_D3Q19) return fail(SC_EINVAL, "the E6 stencil needs D3Q19");
  if (p->psi_self != SC_PSI_N && p->psi_self != SC_PSI_EXP) return fail(SC_EINVAL, "unknown psi %d", p->psi_self);
  if (!isfinite(p->G) || !isfinite(p->G_self[0]) || !isfinite(p->G_self[1]))
    return fail(SC_EINVAL, "couplings must be finite");
  return SC_OK;
}

sc_status scgb::validate_profile_request(const sc_params *p, int32_t kind, const double centre[3], double bin_width,
                                         int32_t nbins, int32_t max_bins) {
  if (kind < SC_PROFILE_RADIAL || kind > SC_PROFILE_AXIS_X) return fail(SC_EINVAL, "unknown profile kind %d", kind);
  if (nbins < 1 || nbins > max_bins) return fail(SC_EINVAL, "nbins must be in [1, %d]", max_bins);
  if (kind == SC_PROFILE_AXIS_X && nbins > p->nx)
    return fail(SC_EINVAL, "the x-axis line has one row per site: nbins must be <= nx (%d)", p->nx);
  if (kind == SC_PROFILE_RADIAL && !(bin_width > 0.0 && isfinite(bin_width)))
    return fail(SC_EINVAL, "bin_width must be finite and > 0");
  for (int m = 0; m < 3; ++m)
    if (!isfinite(centre[m])) return fail(SC_EINVAL, "centre must be finite");
  return SC_OK;
}

ProfileArgs scgb::profile_args(const sc_params *p, int32_t kind, const double centre[3], double bin_width,
                               int32_t nbins) {
  ProfileArgs pa;
  pa.kind = kind;
  for (int m = 0; m < 3; ++m) pa.centre[m] = centre[m];
  pa.bin_width = bin_width;
  pa.nbins = nbins;
  pa.dim = (p->lattice == SC_D3Q19 && p->nz > 1) ? 3 : 2;
  pa.chunk = 0;
  return pa;
}

struct sc_ctx {
  sc_params p;
  int64_t N;
  int Q;
  cudaStream_t stream;
  char *ws;
  Layout L;
  int cur;  // buffer holding the current state
  int tile_y, tile_z;
  int staged, stages, blocks_per_sm;
  int zbal_k, zbal_rem, zbal_cols, zbal_cols_x;  // balanced z split of the staged kernel (zbal_k > 0)
  double nbar[2], psibar[2];
  double scale[2][19], inv_scale[2][19];
  int64_t launches;
  int64_t steps;
  int64_t fields_at;  // step count the FP64 fields were computed at (-1: stale)
  int in_batch;       // stepped by a batch (sc_step refuses)
  // kGraphSteps consecutive step launches from buffer 0, captured once on a private
  // stream and replayed on the context's stream (graph_failed: capture not possible,
  // plain launches only)
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t graph_exec;
  int graph_failed;
};

struct sc_batch {
  int n;
  sc_ctx **ctx;
  cudaStream_t stream;
  void *args_dev;     // StepArgs<CT>[n] (parity 0: buffer 0 -> buffer 1)
  int4 *items_dev;    // (lattice, bx, by, bz) per block
  int nitems;
  int tile_y;
  int staged;         // members step with the staged kernel
  char *retired;      // retired[k]: member k is no longer stepped
  int active;         // members still stepped
  const void *kernel;
  size_t smem;
  // the persistent form of the staged batch (one cooperative launch runs kGraphSteps steps of every
  // member; nullptr when the batch is not staged or the device has no cooperative launch)
  const void *pkernel;
  size_t psmem;
  int pgrid;           // blocks of a persistent launch: the work items, at most the co-resident blocks
  unsigned *counter;   // its grid-barrier counter and kGraphSteps ticket counters (device, zeroed
                       // before every launch)
  int persist_off;     // per-step launches requested (sc_batch_set_persistent(b, 0))
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int64_t steps, launches;
};

namespace {

unsigned int *status_word(sc_ctx *c) { return reinterpret_cast<unsigned int *>(c->ws + c->L.off_status); }
double *status_scalars(sc_ctx *c) { return reinterpret_cast<double *>(c->ws + c->L.off_status + 256); }
double *analysis_rows(sc_ctx *c) { return reinterpret_cast<double *>(c->ws + c->L.off_analysis); }
double *analysis_pio(sc_ctx *c) { return analysis_rows(c) + (size_t)kMaxProfileBins * 6; }
double *fields_of(sc_ctx *c) { return reinterpret_cast<double *>(c->ws + c->L.off_fields); }
double *partial_of(sc_ctx *c) { return reinterpret_cast<double *>(c->ws + c->L.off_partial); }

PopArgs pop_args(sc_ctx *c, int buf) {
  PopArgs a;
  a.buf = c->ws + c->L.off_pop[buf];
  a.nref = c->L.ref_bytes ? reinterpret_cast<float2 *>(c->ws + c->L.off_ref[buf]) : nullptr;
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.nz = c->p.nz;
  a.N = c->N;
  for (int J = 0; J < 2; ++J) {
    a.nbar[J] = c->nbar[J];
    for (int i = 0; i < 19; ++i) {
      a.scale[J][i] = c->scale[J][i];
      a.inv_scale[J][i] = c->inv_scale[J][i];
    }
  }
  return a;
}

ForceParams force_params(const sc_ctx *c) {
  ForceParams f;
  f.G = c->p.G;
  f.G_self[0] = c->p.G_self[0];
  f.G_self[1] = c->p.G_self[1];
  f.nx = c->p.nx;
  f.ny = c->p.ny;
  f.nz = c->p.nz;
  f.N = c->N;
  return f;
}

int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

// Dispatch on (lattice, storage) for the population-access kernels.
#define SC_POP_DISPATCH(ctx, KERNEL, grid, block, smem, ...)                                             \
  do {                                                                                                    \
    const int lat_ = (ctx)->p.lattice, st_ = (ctx)->p.storage;                                           \
    if (lat_ == SC_D3Q19) {                                                                               \
      if (st_ == SC_STORE_F32) KERNEL<kD3Q19, float><<<grid, block, smem, (ctx)->stream>>>(__VA_ARGS__);  \
      if (st_ == SC_STORE_F16) KERNEL<kD3Q19, __half><<<grid, block, smem, (ctx)->stream>>>(__VA_ARGS__); \
      if (st_ == SC_STORE_BF16)                                                                           \
        KERNEL<kD3Q19, __nv_bfloat16><<<grid, block, smem, (ctx)->stream>>>(__VA_ARGS__);                 \
      if (st_ == SC_STORE_F64) KERNEL<kD3Q19, double><<<grid, block, smem, (ctx)->stream>>>(__VA_ARGS__); \
    } else {                                                                                              \
      if (st_ == SC_STORE_F32) KERNEL<kD2Q9, float><<<grid, block, smem, (ctx)->stream>>>(__VA_ARGS__);   \
      if (st_ == SC_STORE_F16) KERNEL<kD2Q9, __half><<<grid, block, smem, (ctx)->stream>>>(__VA_ARGS__);  \
      if (st_ == SC_STORE_BF16)                                                                           \
        KERNEL<kD2Q9, __nv_bfloat16><<<grid, block, smem, (ctx)->stream>>>(__VA_ARGS__);                  \
      if (st_ == SC_STORE_F64) KERNEL<kD2Q9, double><<<grid, block, smem, (ctx)->stream>>>(__VA_ARGS__);  \
    }                                                                                                     \
  } while (0)

// FP64 density / pseudopotential fields of the current state (cached per step count).
sc_status ensure_fields(sc_ctx *c) {
  if (c->fields_at == c->steps) return SC_OK;
  PopArgs a = pop_args(c, c->cur);
  SC_POP_DISPATCH(c, fields_kernel, grid_for(c->N, 256), 256, 0, a, c->p.psi_self, fields_of(c));
  SC_CUDA(cudaGetLastError());
  c->fields_at = c->steps;
  return SC_OK;
}

template <class CT>
P2<CT> pair(double a, double b) {
  P2<CT> p;
  p.x = CT(a);
  p.y = CT(b);
  return p;
}

template <class CT>
StepArgs<CT> step_args(sc_ctx *c) {
  StepArgs<CT> a;
  memset(&a, 0, sizeof(a));
  a.src = c->ws + c->L.off_pop[c->cur];
  a.dst = c->ws + c->L.off_pop[1 - c->cur];
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.nz = c->p.nz;
  a.tile_z = c->tile_z;
  a.N = c->N;
  const double cs2 = 1.0 / 3.0;
  a.nbar = pair<CT>(c->nbar[0], c->nbar[1]);
  a.omega = pair<CT>(1.0 / c->p.tau[0], 1.0 / c->p.tau[1]);
  a.guo = pair<CT>(1.0 - 0.5 / c->p.tau[0], 1.0 - 0.5 / c->p.tau[1]);
  a.gself = pair<CT>(-c->p.G_self[0] * cs2, -c->p.G_self[1] * cs2);
  a.psibar = pair<CT>(c->psibar[0], c->psibar[1]);
  a.scale = pair<CT>(c->scale[0][0], c->scale[1][0]);
  a.inv_scale = pair<CT>(c->inv_scale[0][0], c->inv_scale[1][0]);
  a.gcross = CT(-c->p.G * cs2);
  a.self_on = (c->p.G_self[0] != 0.0 || c->p.G_self[1] != 0.0) ? 1 : 0;
  a.tau_one = tau_one(&c->p) ? 1 : 0;
  a.psi_exp = c->p.psi_self == SC_PSI_EXP ? 1 : 0;
  a.err = status_word(c);
  a.nsrc = c->L.ref_bytes ? reinterpret_cast<const float2 *>(c->ws + c->L.off_ref[c->cur]) : nullptr;
  a.ndst = c->L.ref_bytes ? reinterpret_cast<float2 *>(c->ws + c->L.off_ref[1 - c->cur]) : nullptr;
  a.zbal_k = c->zbal_k;
  a.zbal_rem = c->zbal_rem;
  a.zbal_cols = c->zbal_cols;
  a.zbal_cols_x = c->zbal_cols_x;
  return a;
}

// Target z-chunk of the generic kernel's balanced split, in planes (same-box comparison, FP32
// and FP16, E4 and E6: targets 16, 24 and 32 pick one full wave for the 64 x 64 x 256 slab and
// 96^3, where all agree; at 128^3 two waves of 13-14 planes (target 16) beat one of 27 by 2 to
// 9 %.  Against the earlier fixed 16..32-plane chunks: E6 slab 10.5 -> 11.4 GLUPS, E6 128^3
// 8.2 -> 11.3, E6 96^3 8.9 -> 10.5).
constexpr int kGenericTargetChunk = 16;

// z-chunking of a D3Q19 lattice when tile_z is left to the library.  Staged kernel: 128 or
// 64 planes where that grid still fills eight waves of the GPU.  Either kernel: 32 planes
// where a 32-plane grid fills four waves, otherwise a balanced z split: the grid is exactly
// waves x (SMs x resident blocks per SM) blocks, with waves chosen for z-chunks of about
// a target chunk length (wave count rounded to nearest), and every column of 32 x tile_y sites
// is cut into K or K + 1 equal z-chunks.  A fixed tile_z instead leaves a partly empty last
// wave whenever the block count is not a multiple of the resident slots (staged, 128^3: 256
// blocks of 32 planes for 304 slots; generic E6, 128^3: 320 blocks of 26 planes for 304).
sc_status plan_z_split(sc_ctx *c) {
  // Staged FP32, same box: 18 planes beat 12 and 36 at 128^3 (16.5 against 15.9 and 15.1 GLUPS)
  // and tie with 36 at 160^3 and 192^3.  Staged 16-bit storage is issue-bound, so the two re-summed
  // z-halo planes per chunk weigh more: 36 planes beat 18 by 2-3 % at 160^3 and 192^3 (equal at
  // 128^3, one wave either way).  The generic kernel re-sums 2 HALO z-halo planes per chunk from
  // L2 instead of a staged window.
  const int target_chunk = !c->staged ? kGenericTargetChunk : (is_16bit(c->p.storage) ? 36 : 18);
  int dev = 0, sms = 0, occ = 0;
  const bool self_on = has_self(&c->p), t1 = tau_one(&c->p);
  const int lat = c->p.lattice == SC_D3Q19 ? kD3Q19 : kD2Q9, sten = c->p.stencil == SC_FORCE_E6 ? kE6 : kE4;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && c->staged) {
    switch (c->p.storage) {
      case SC_STORE_F32: e = staged_occupancy_f32(c->tile_y, c->stages, c->blocks_per_sm, self_on, t1, &occ); break;
      case SC_STORE_F16: e = staged_occupancy_f16(c->tile_y, c->stages, c->blocks_per_sm, self_on, t1, &occ); break;
      case SC_STORE_BF16: e = staged_occupancy_bf16(c->tile_y, c->stages, c->blocks_per_sm, self_on, t1, &occ); break;
      default: e = staged_occupancy_f64(c->tile_y, c->stages, c->blocks_per_sm, self_on, t1, &occ); break;
    }
  } else if (e == cudaSuccess) {
    switch (c->p.storage) {
      case SC_STORE_F32: e = generic_occupancy_f32(lat, sten, c->tile_y, t1, &occ); break;
      case SC_STORE_F16: e = generic_occupancy_f16(lat, sten, c->tile_y, t1, &occ); break;
      case SC_STORE_BF16: e = generic_occupancy_bf16(lat, sten, c->tile_y, t1, &occ); break;
      default: e = generic_occupancy_f64(lat, sten, c->tile_y, t1, &occ); break;
    }
  }
  if (e != cudaSuccess) return fail(SC_ECUDA, "occupancy of the step kernel: %s", cudaGetErrorString(e));
  const int64_t cols_x = (c->p.nx + 31) / 32, cols = cols_x * ((c->p.ny + c->tile_y - 1) / c->tile_y);
  const int64_t nz = c->p.nz, slots = (int64_t)sms * (occ > 0 ? occ : 1);
  // deep grids: the longest z-chunks (fewer re-summed z-halo planes per site) that still leave
  // eight waves (512^3: 16-bit +3.8 % with 128 planes over 32; 256^3 stays at 32)
  if (c->staged) {
    for (int tz : {128, 64}) {
      if (cols * ((nz + tz - 1) / tz) >= 8 * slots) {
        c->tile_z = (int)(tz < nz ? tz : nz);
        return SC_OK;
      }
    }
  }
  const int64_t fixed_blocks = cols * ((nz + c->tile_z - 1) / c->tile_z);
  if (fixed_blocks >= 4 * slots) return SC_OK;  // many waves: the plain grid's last-wave loss is small
  int64_t waves = (2 * cols * nz + slots * target_chunk) / (2 * slots * target_chunk);  // rounded
  if (waves < 1) waves = 1;
  int64_t G = slots * waves;
  const int64_t gmax = cols * (nz / 4 > 1 ? nz / 4 : 1);  // chunks of 4 planes or more
  if (G > gmax) G = gmax;
  if (G < cols || G > (int64_t(1) << 31) - 1) return SC_OK;  // more columns than slots: plain grid
  c->zbal_k = (int)(G / cols);
  c->zbal_rem = (int)(G % cols);
  c->zbal_cols = (int)cols;
  c->zbal_cols_x = (int)cols_x;
  return SC_OK;
}

sc_status launch_one_step(sc_ctx *c) {
  StepLaunch l;
  l.lattice = c->p.lattice == SC_D3Q19 ? kD3Q19 : kD2Q9;
  l.stencil = c->p.stencil == SC_FORCE_E6 ? kE6 : kE4;
  l.tile_y = c->tile_y;
  l.staged = c->staged;
  l.stages = c->stages;
  l.blocks_per_sm = c->blocks_per_sm;
  l.grid = dim3((c->p.nx + 31) / 32, (c->p.ny + c->tile_y - 1) / c->tile_y, (c->p.nz + c->tile_z - 1) / c->tile_z);
  l.stream = c->stream;
  cudaError_t e;
  switch (c->p.storage) {
    case SC_STORE_F32: e = launch_step_f32(l, step_args<float>(c)); break;
    case SC_STORE_F16: e = launch_step_f16(l, step_args<float>(c)); break;
    case SC_STORE_BF16: e = launch_step_bf16(l, step_args<float>(c)); break;
    default: e = launch_step_f64(l, step_args<double>(c)); break;
  }
  if (e != cudaSuccess) return fail(SC_ECUDA, "step kernel launch: %s", cudaGetErrorString(e));
  c->cur = 1 - c->cur;
  c->launches++;
  c->steps++;
  return SC_OK;
}

// Deterministic sums / maxima of the two initial fields.
sc_status init_reductions(sc_ctx *c, const double *nA0, const double *nB0, double *mean, double *maxdev) {
  const int blocks = grid_for(c->N, 256) < kMaxPartialBlocks ? grid_for(c->N, 256) : kMaxPartialBlocks;
  double *part = partial_of(c);
  double *sc = status_scalars(c);
  min2_partial_kernel<<<blocks, 256, 0, c->stream>>>(nA0, nB0, c->N, part);
  SC_CUDA(cudaGetLastError());
  double *mins = (double *)malloc(sizeof(double) * blocks);
  if (!mins) return fail(SC_ENOMEM, "host allocation failed");
  cudaError_t e = cudaMemcpyAsync(mins, part, sizeof(double) * blocks, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free(mins);
    return fail(SC_ECUDA, "reading initial-field minima: %s", cudaGetErrorString(e));
  }
  bool bad = false;
  for (int k = 0; k < blocks; ++k) bad |= !(mins[k] > 0.0);
  free(mins);
  if (bad) return fail(SC_EINVAL, "initial densities must be finite and > 0");
  sum2_partial_kernel<<<blocks, 256, 0, c->stream>>>(nA0, nB0, c->N, part);
  totals_finalize_kernel<<<1, 32, 0, c->stream>>>(part, blocks, 2, sc);
  SC_CUDA(cudaGetLastError());
  SC_CUDA(cudaMemcpyAsync(mean, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SC_CUDA(cudaStreamSynchronize(c->stream));
  mean[0] /= (double)c->N;
  mean[1] /= (double)c->N;
  maxdev_partial_kernel<<<blocks, 256, 0, c->stream>>>(nA0, nB0, c->N, mean[0], mean[1], part);
  SC_CUDA(cudaGetLastError());
  double *md = (double *)malloc(sizeof(double) * 2 * blocks);
  if (!md) return fail(SC_ENOMEM, "host allocation failed");
  e = cudaMemcpyAsync(md, part, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free(md);
    return fail(SC_ECUDA, "reading initial-field deviations: %s", cudaGetErrorString(e));
  }
  maxdev[0] = maxdev[1] = 0.0;
  for (int k = 0; k < blocks; ++k) {
    maxdev[0] = fmax(maxdev[0], md[2 * k]);
    maxdev[1] = fmax(maxdev[1], md[2 * k + 1]);
  }
  free(md);
  return SC_OK;
}

double lattice_w(int lattice, int i) {
  if (lattice == SC_D3Q19) return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

}  // namespace

extern "C" {

size_t sc_workspace_bytes(const sc_params *params) {
  if (validate(params) != SC_OK) return 0;
  return layout_of(params).total;
}

sc_status sc_create(const sc_params *params, const double *nA0, const double *nB0, void *workspace, size_t ws_bytes,
                    void *stream, sc_ctx **out) {
  if (!out) return fail(SC_EINVAL, "out is NULL");
  *out = nullptr;
  sc_status st = validate(params);
  if (st != SC_OK) return st;
  if (!nA0 || !nB0 || !workspace) return fail(SC_EINVAL, "initial fields and workspace must be non-NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return fail(SC_EINVAL, "workspace must be 256-byte aligned");
  Layout L = layout_of(params);
  if (ws_bytes < L.total) return fail(SC_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
  sc_ctx *c = new (std::nothrow) sc_ctx;
  if (!c) return fail(SC_ENOMEM, "host allocation failed");
  memset(c, 0, sizeof(*c));
  c->p = *params;
  c->N = (int64_t)params->nx * params->ny * params->nz;
  c->Q = q_of(params);
  c->stream = static_cast<cudaStream_t>(stream);
  c->ws = static_cast<char *>(workspace);
  c->L = L;
  c->cur = 0;
  c->tile_y = default_tile_y(params);
  c->tile_z = default_tile_z(params);
  c->staged = use_staged(params) ? 1 : 0;
  c->stages = effective_stages(params, c->tile_y);
  c->blocks_per_sm = effective_blocks_per_sm(params, c->tile_y);
  c->fields_at = -1;
  if (params->tile_z == 0 && params->lattice == SC_D3Q19) {
    st = plan_z_split(c);
    if (st != SC_OK) {
      delete c;
      return st;
    }
  }
  double mean[2], maxdev[2];
  cudaError_t e = cudaMemsetAsync(c->ws + L.off_status, 0, kStatusBytes, c->stream);
  if (e != cudaSuccess) {
    delete c;
    return fail(SC_ECUDA, "clearing the status word: %s", cudaGetErrorString(e));
  }
  st = init_reductions(c, nA0, nB0, mean, maxdev);
  if (st != SC_OK) {
    delete c;
    return st;
  }
  for (int J = 0; J < 2; ++J) {
    c->nbar[J] = mean[J];
    c->psibar[J] = params->psi_self == SC_PSI_EXP ? exp(-1.0 / mean[J]) : mean[J];
    double s = 1.0;
    if (params->storage == SC_STORE_F16) {
      // stored values are deviations from each site's own rest equilibrium, of order
      // w_i n |u| (plus the non-equilibrium part); take 0.1 w_0 n_max (w_0 the largest
      // weight) as their scale and the largest power of two keeping it <= 2^10 (FP16 max
      // 65504: x64 headroom; the smallest weight is 1/12 of w_0, far from underflow)
      const double m = 0.1 * lattice_w(params->lattice, 0) * fmax(mean[J] + maxdev[J], 1e-3);
      s = ldexp(1.0, (int)floor(log2(1024.0 / m)));
    }
    for (int i = 0; i < 19; ++i) {
      c->scale[J][i] = s;
      c->inv_scale[J][i] = 1.0 / s;
    }
  }
  PopArgs a = pop_args(c, 0);
  SC_POP_DISPATCH(c, pop_kernel, grid_for(c->N, 256), 256, 0, a, 0, nA0, nB0, nullptr);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    delete c;
    return fail(SC_ECUDA, "initialising populations: %s", cudaGetErrorString(e));
  }
  *out = c;
  return SC_OK;
}

namespace {
constexpr int kStepGraphSteps = 32;  // steps per replay of a context's step graph (even: parity kept)

// Capture kStepGraphSteps step launches (starting from buffer 0) on a private stream and
// instantiate them.  Any failure leaves the context on plain launches (graph_failed).
void build_step_graph(sc_ctx *c) {
  cudaStream_t user = c->stream;
  const int64_t launches = c->launches, steps = c->steps, fields_at = c->fields_at;
  bool ok = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) {
    c->stream = c->cap_stream;
    ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
      for (int t = 0; t < kStepGraphSteps && ok; ++t) ok = launch_one_step(c) == SC_OK;
      cudaGraph_t g = nullptr;
      const bool ended = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess;
      ok = ok && ended && g;
      if (ok) {
        c->graph = g;
        ok = cudaGraphInstantiate(&c->graph_exec, g, 0) == cudaSuccess;
      } else if (g) {
        cudaGraphDestroy(g);
      }
    }
  }
  c->stream = user;
  c->cur = 0;
  c->launches = launches;
  c->steps = steps;
  c->fields_at = fields_at;
  if (!ok) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_failed = 1;
    cudaGetLastError();  // the capture's error is not the caller's
  }
}
}  // namespace

sc_status sc_step(sc_ctx *c, int64_t nsteps) {
  if (!c) return fail(SC_EINVAL, "ctx is NULL");
  if (c->in_batch) return fail(SC_EINVAL, "this context belongs to a batch: step it with sc_batch_step");
  if (nsteps < 0) return fail(SC_EINVAL, "nsteps must be >= 0");
  while (nsteps > 0) {
    // runs of kStepGraphSteps from buffer 0 replay the step graph (built on first use,
    // once the kernel has launched normally)
    if (c->cur == 0 && nsteps >= kStepGraphSteps && c->launches >= 2 && !c->graph_failed) {
      if (!c->graph_exec) build_step_graph(c);
      if (c->graph_exec) {
        SC_CUDA(cudaGraphLaunch(c->graph_exec, c->stream));
        c->launches += kStepGraphSteps;
        c->steps += kStepGraphSteps;
        nsteps -= kStepGraphSteps;
        continue;
      }
    }
    sc_status st = launch_one_step(c);
    if (st != SC_OK) return st;
    nsteps -= 1;
  }
  return SC_OK;
}

sc_status sc_moments(sc_ctx *c, double *nA, double *nB, double *u) {
  if (!c || !nA || !nB) return fail(SC_EINVAL, "ctx, nA and nB must be non-NULL");
  sc_status st = ensure_fields(c);
  if (st != SC_OK) return st;
  double *F = fields_of(c);
  SC_CUDA(cudaMemcpyAsync(nA, F, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  SC_CUDA(cudaMemcpyAsync(nB, F + c->N, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  if (u) {
    PopArgs a = pop_args(c, c->cur);
    ForceParams fp = force_params(c);
    const int g = grid_for(c->N, 128);
    const int lat = c->p.lattice, sten = c->p.stencil, s = c->p.storage;
#define SC_VEL(LAT, STEN, ST) velocity_kernel<LAT, STEN, ST><<<g, 128, 0, c->stream>>>(a, fp, F, u)
#define SC_VEL_ST(LAT, STEN)                    \
  do {                                          \
    if (s == SC_STORE_F32) SC_VEL(LAT, STEN, float);         \
    if (s == SC_STORE_F16) SC_VEL(LAT, STEN, __half);        \
    if (s == SC_STORE_BF16) SC_VEL(LAT, STEN, __nv_bfloat16); \
    if (s == SC_STORE_F64) SC_VEL(LAT, STEN, double);        \
  } while (0)
    if (lat == SC_D3Q19 && sten == SC_FORCE_E4) SC_VEL_ST(kD3Q19, kE4);
    if (lat == SC_D3Q19 && sten == SC_FORCE_E6) SC_VEL_ST(kD3Q19, kE6);
    if (lat == SC_D2Q9) SC_VEL_ST(kD2Q9, kE4);
#undef SC_VEL_ST
#undef SC_VEL
    SC_CUDA(cudaGetLastError());
  }
  return SC_OK;
}

sc_status sc_velocity_change(sc_ctx *c, double *u_prev, double *out) {
  if (!c || !u_prev || !out) return fail(SC_EINVAL, "ctx, u_prev and out must be non-NULL");
  sc_status st = ensure_fields(c);
  if (st != SC_OK) return st;
  PopArgs a = pop_args(c, c->cur);
  ForceParams fp = force_params(c);
  const double *F = fields_of(c);
  double *part = partial_of(c);
  const int blocks = grid_for(c->N, 256) < kMaxPartialBlocks ? grid_for(c->N, 256) : kMaxPartialBlocks;
  const int lat = c->p.lattice, sten = c->p.stencil, s = c->p.storage;
#define SC_DU(LAT, STEN, ST) \
  velocity_change_partial_kernel<LAT, STEN, ST><<<blocks, 256, 0, c->stream>>>(a, fp, F, u_prev, part)
#define SC_DU_ST(LAT, STEN)                                   \
  do {                                                        \
    if (s == SC_STORE_F32) SC_DU(LAT, STEN, float);           \
    if (s == SC_STORE_F16) SC_DU(LAT, STEN, __half);          \
    if (s == SC_STORE_BF16) SC_DU(LAT, STEN, __nv_bfloat16);  \
    if (s == SC_STORE_F64) SC_DU(LAT, STEN, double);          \
  } while (0)
  if (lat == SC_D3Q19 && sten == SC_FORCE_E4) SC_DU_ST(kD3Q19, kE4);
  if (lat == SC_D3Q19 && sten == SC_FORCE_E6) SC_DU_ST(kD3Q19, kE6);
  if (lat == SC_D2Q9) SC_DU_ST(kD2Q9, kE4);
#undef SC_DU_ST
#undef SC_DU
  finalize_measure_kernel<<<1, 32, 0, c->stream>>>(part, blocks, 0, 1.0 / double(c->N), out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

sc_status sc_centre_of_mass(sc_ctx *c, int32_t component, double background, double *out) {
  if (!c || !out) return fail(SC_EINVAL, "ctx and out must be non-NULL");
  if (component != 0 && component != 1) return fail(SC_EINVAL, "component must be 0 (A) or 1 (B)");
  if (!isfinite(background)) return fail(SC_EINVAL, "background must be finite");
  sc_status st = ensure_fields(c);
  if (st != SC_OK) return st;
  const int blocks = grid_for(c->N, 256) < kMaxPartialBlocks ? grid_for(c->N, 256) : kMaxPartialBlocks;
  double *part = partial_of(c);
  com_partial_kernel<<<blocks, 256, 0, c->stream>>>(fields_of(c) + (int64_t)component * c->N, c->p.nx, c->p.ny, c->N,
                                                    background, part);
  finalize_measure_kernel<<<1, 32, 0, c->stream>>>(part, blocks, 1, 1.0, out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

sc_status sc_get_populations(sc_ctx *c, double *f) {
  if (!c || !f) return fail(SC_EINVAL, "ctx and f must be non-NULL");
  PopArgs a = pop_args(c, c->cur);
  SC_POP_DISPATCH(c, pop_kernel, grid_for(c->N, 256), 256, 0, a, 2, nullptr, nullptr, f);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

sc_status sc_set_populations(sc_ctx *c, const double *f) {
  if (!c || !f) return fail(SC_EINVAL, "ctx and f must be non-NULL");
  PopArgs a = pop_args(c, c->cur);
  SC_POP_DISPATCH(c, pop_kernel, grid_for(c->N, 256), 256, 0, a, 1, nullptr, nullptr, const_cast<double *>(f));
  SC_CUDA(cudaGetLastError());
  c->fields_at = -1;
  return SC_OK;
}

size_t sc_state_bytes(const sc_ctx *c) { return c ? c->L.pop_bytes + c->L.ref_bytes : 0; }

sc_status sc_get_state(sc_ctx *c, void *dst, size_t bytes) {
  if (!c || !dst) return fail(SC_EINVAL, "ctx and dst must be non-NULL");
  const size_t need = c->L.pop_bytes + c->L.ref_bytes;
  if (bytes != need) return fail(SC_EINVAL, "state is %zu bytes, got %zu", need, bytes);
  SC_CUDA(cudaMemcpyAsync(dst, c->ws + c->L.off_pop[c->cur], c->L.pop_bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (c->L.ref_bytes)
    SC_CUDA(cudaMemcpyAsync(static_cast<char *>(dst) + c->L.pop_bytes, c->ws + c->L.off_ref[c->cur], c->L.ref_bytes,
                            cudaMemcpyDeviceToDevice, c->stream));
  return SC_OK;
}

sc_status sc_set_state(sc_ctx *c, const void *src, size_t bytes) {
  if (!c || !src) return fail(SC_EINVAL, "ctx and src must be non-NULL");
  const size_t need = c->L.pop_bytes + c->L.ref_bytes;
  if (bytes != need) return fail(SC_EINVAL, "state is %zu bytes, got %zu", need, bytes);
  SC_CUDA(cudaMemcpyAsync(c->ws + c->L.off_pop[c->cur], src, c->L.pop_bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (c->L.ref_bytes)
    SC_CUDA(cudaMemcpyAsync(c->ws + c->L.off_ref[c->cur], static_cast<const char *>(src) + c->L.pop_bytes,
                            c->L.ref_bytes, cudaMemcpyDeviceToDevice, c->stream));
  c->fields_at = -1;
  return SC_OK;
}

sc_status sc_pressure_profile(sc_ctx *c, int32_t kind, const double centre[3], double bin_width, int32_t nbins,
                              double *out) {
  if (!c || !out || !centre) return fail(SC_EINVAL, "ctx, centre and out must be non-NULL");
  sc_status st = validate_profile_request(&c->p, kind, centre, bin_width, nbins, kMaxProfileBins);
  if (st != SC_OK) return st;
  st = ensure_fields(c);
  if (st != SC_OK) return st;
  SC_CUDA(launch_profile(c->p.lattice, c->p.stencil, force_params(c), profile_args(&c->p, kind, centre, bin_width, nbins),
                         StoredFields{fields_of(c), c->N}, partial_of(c), (int64_t)(kPartialBytes / sizeof(double)),
                         kMaxPartialBlocks, out, c->stream));
  return SC_OK;
}

sc_status sc_bulk_pressure_at(sc_ctx *c, const int32_t node[3], double *out) {
  if (!c || !node || !out) return fail(SC_EINVAL, "ctx, node and out must be non-NULL");
  const int nn[3] = {c->p.nx, c->p.ny, c->p.nz};
  for (int m = 0; m < 3; ++m)
    if (node[m] < 0 || node[m] >= nn[m]) return fail(SC_EINVAL, "node outside the lattice");
  sc_status st = ensure_fields(c);
  if (st != SC_OK) return st;
  const int64_t s = (int64_t)node[0] + (int64_t)c->p.nx * (node[1] + (int64_t)c->p.ny * node[2]);
  bulk_pressure_kernel<<<1, 32, 0, c->stream>>>(force_params(c), fields_of(c), s, out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

sc_status sc_sigma_minimum(const double *rows, int32_t nbins, const double *P_in_out, int32_t dim, double R_lo,
                           double R_hi, double R_step, double *out, void *stream) {
  if (!rows || !P_in_out || !out) return fail(SC_EINVAL, "rows, P_in_out and out must be non-NULL");
  if (nbins < 2) return fail(SC_EINVAL, "need at least two profile rows");
  if (dim != 2 && dim != 3) return fail(SC_EINVAL, "dim must be 2 or 3");
  if (!(R_lo > 0.0) || !(R_hi > R_lo) || !(R_step > 0.0) || (R_hi - R_lo) / R_step > 1e7)
    return fail(SC_EINVAL, "need 0 < R_lo < R_hi, R_step > 0 and at most 1e7 grid points");
  sigma_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(rows, nbins, P_in_out, dim, R_lo, R_hi, R_step, out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

sc_status sc_surface_of_tension(sc_ctx *c, int32_t kind, const double centre[3], double bin_width, int32_t nbins,
                                double R_lo, double R_hi, double R_step, double *out, double *rows) {
  if (!c || !out) return fail(SC_EINVAL, "ctx and out must be non-NULL");
  if (kind != SC_PROFILE_RADIAL && kind != SC_PROFILE_AXIS_X)
    return fail(SC_EINVAL, "the surface of tension takes a radial or an x-axis profile, not kind %d", kind);
  const int dim = (c->p.lattice == SC_D3Q19 && c->p.nz > 1) ? 3 : 2;
  const int nn[3] = {c->p.nx, c->p.ny, c->p.nz};
  double ctr[3];
  for (int m = 0; m < 3; ++m) ctr[m] = centre ? centre[m] : (double)(nn[m] / 2);
  if (kind == SC_PROFILE_AXIS_X) bin_width = 1.0;
  if (nbins == 0) {
    // the largest sphere (circle) inside the box, or half the x axis
    int half = kind == SC_PROFILE_AXIS_X ? nn[0] : (dim == 3 ? std::min(nn[0], std::min(nn[1], nn[2]))
                                                             : std::min(nn[0], nn[1]));
    nbins = kind == SC_PROFILE_AXIS_X ? half / 2 : (int32_t)(half / 2 / bin_width);
  }
  if (nbins < 2) return fail(SC_EINVAL, "need at least two profile rows");
  sc_status st = validate_profile_request(&c->p, kind, ctr, bin_width, nbins, kMaxProfileBins);
  if (st != SC_OK) return st;
  const double r_max = nbins * bin_width;
  if (R_step == 0.0) R_step = 0.01;
  if (R_lo == 0.0) R_lo = R_step;
  if (R_hi == 0.0) R_hi = r_max;
  if (!(R_lo > 0.0) || !(R_hi > R_lo) || !(R_step > 0.0) || (R_hi - R_lo) / R_step > 1e7)
    return fail(SC_EINVAL, "need 0 < R_lo < R_hi, R_step > 0 and at most 1e7 grid points");
  double *r = rows ? rows : analysis_rows(c);
  st = sc_pressure_profile(c, kind, ctr, bin_width, nbins, r);
  if (st != SC_OK) return st;
  // P_in at the centre node, P_out at the far corner (section 4)
  int32_t in_node[3], out_node[3];
  for (int m = 0; m < 3; ++m) {
    const int k = (int)floor(ctr[m] + 0.5);
    in_node[m] = ((k % nn[m]) + nn[m]) % nn[m];
    out_node[m] = nn[m] - 1;
  }
  double *pio = analysis_pio(c);
  st = sc_bulk_pressure_at(c, in_node, pio);
  if (st == SC_OK) st = sc_bulk_pressure_at(c, out_node, pio + 1);
  if (st != SC_OK) return st;
  return sc_sigma_minimum(r, nbins, pio, dim, R_lo, R_hi, R_step, out, c->stream);
}

sc_status sc_diagnostics(sc_ctx *c, double *u_prev, int32_t component, double background, double *out) {
  if (!c || !out) return fail(SC_EINVAL, "ctx and out must be non-NULL");
  if (component < -1 || component > 1) return fail(SC_EINVAL, "component must be -1 (none), 0 (A) or 1 (B)");
  if (component >= 0 && !isfinite(background)) return fail(SC_EINVAL, "background must be finite");
  sc_status st = sc_totals(c, out);
  if (st != SC_OK) return st;
  if (u_prev) {
    st = sc_velocity_change(c, u_prev, out + 5);
    if (st != SC_OK) return st;
  } else {
    SC_CUDA(cudaMemsetAsync(out + 5, 0xff, sizeof(double), c->stream));  // all-ones bits: a NaN
  }
  if (component >= 0) return sc_centre_of_mass(c, component, background, out + 6);
  SC_CUDA(cudaMemsetAsync(out + 6, 0xff, 4 * sizeof(double), c->stream));
  return SC_OK;
}

sc_status sc_sigma0_flat(const double *rows, int32_t nbins, double *out, void *stream) {
  if (!rows || !out) return fail(SC_EINVAL, "rows and out must be non-NULL");
  if (nbins < 2) return fail(SC_EINVAL, "need at least two planes");
  sigma0_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(rows, nbins, out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

sc_status sc_curvature_fit(const double *Rs, const double *sigma_s, int32_t n, int32_t order, const double *sigma0,
                           double *out, void *stream) {
  if (!Rs || !sigma_s || !out) return fail(SC_EINVAL, "Rs, sigma_s and out must be non-NULL");
  if (order != 1 && order != 2) return fail(SC_EINVAL, "order must be 1 or 2");
  const int unknowns = order + (sigma0 ? 0 : 1);
  if (n < unknowns || n > (1 << 20)) return fail(SC_EINVAL, "need %d to 2^20 droplets, got %d", unknowns, n);
  curvature_fit_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(Rs, sigma_s, n, order, sigma0, out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

sc_status sc_totals(sc_ctx *c, double *out) {
  if (!c || !out) return fail(SC_EINVAL, "ctx and out must be non-NULL");
  const int blocks = grid_for(c->N, 256) < kMaxPartialBlocks ? grid_for(c->N, 256) : kMaxPartialBlocks;
  PopArgs a = pop_args(c, c->cur);
  SC_POP_DISPATCH(c, totals_partial_kernel, blocks, 256, 0, a, partial_of(c));
  totals_finalize_kernel<<<1, 32, 0, c->stream>>>(partial_of(c), blocks, 5, out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

sc_status sc_sync(sc_ctx *c) {
  if (!c) return fail(SC_EINVAL, "ctx is NULL");
  SC_CUDA(cudaStreamSynchronize(c->stream));
  unsigned int w = 0;
  SC_CUDA(cudaMemcpy(&w, status_word(c), sizeof(w), cudaMemcpyDeviceToHost));
  if (w) {
    SC_CUDA(cudaMemset(status_word(c), 0, sizeof(unsigned int)));
    if (w & 2u)
      return fail(SC_ETIMEOUT, "a bounded device-side wait of a step kernel ran out (status 0x%x)", w);
    return fail(SC_ENAN, "a time step met a non-finite density, or a non-positive one with psi = exp(-1/n) "
                         "(status 0x%x)", w);
  }
  return SC_OK;
}

sc_status sc_selftest_wait_timeout(sc_ctx *c, int32_t max_polls) {
  if (!c) return fail(SC_EINVAL, "ctx is NULL");
  if (max_polls < 1 || max_polls > (1 << 20)) return fail(SC_EINVAL, "max_polls must be in [1, 2^20]");
  // the probe's barrier counter: a word of the status area that nothing else uses
  unsigned *counter = reinterpret_cast<unsigned *>(c->ws + c->L.off_status + 128);
  SC_CUDA(launch_barrier_probe(counter, status_word(c), (unsigned)max_polls, c->stream));
  return SC_OK;
}

sc_status sc_run_host(const sc_params *params, const double *nA0, const double *nB0, int64_t nsteps, double *nA,
                      double *nB, void *workspace, size_t ws_bytes, void *stream) {
  sc_status st = validate(params);
  if (st != SC_OK) return st;
  if (!nA0 || !nB0 || !nA || !nB || !workspace) return fail(SC_EINVAL, "buffers must be non-NULL");
  if (nsteps < 0) return fail(SC_EINVAL, "nsteps must be >= 0");
  Layout L = layout_of(params);
  if (ws_bytes < L.total) return fail(SC_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
  const int64_t N = (int64_t)params->nx * params->ny * params->nz;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // stage the initial fields in the (not yet used) FP64 field region
  double *stage = reinterpret_cast<double *>(static_cast<char *>(workspace) + L.off_fields);
  SC_CUDA(cudaMemcpyAsync(stage, nA0, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  SC_CUDA(cudaMemcpyAsync(stage + N, nB0, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  sc_ctx *c = nullptr;
  st = sc_create(params, stage, stage + N, workspace, ws_bytes, stream, &c);
  if (st != SC_OK) return st;
  st = sc_step(c, nsteps);
  if (st == SC_OK) st = ensure_fields(c);
  if (st == SC_OK) {
    cudaError_t e = cudaMemcpyAsync(nA, fields_of(c), sizeof(double) * N, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nB, fields_of(c) + N, sizeof(double) * N, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = fail(SC_ECUDA, "copying densities to the host: %s", cudaGetErrorString(e));
  }
  if (st == SC_OK) st = sc_sync(c);
  sc_destroy(c);
  return st;
}

sc_status sc_run_host_sigma(const sc_params *params, const double *nA0, const double *nB0, int64_t nsteps,
                           const double centre[3], double bin_width, int32_t nbins, double *nA, double *nB,
                           double *result, void *workspace, size_t ws_bytes, void *stream) {
  sc_status st = validate(params);
  if (st != SC_OK) return st;
  if (!nA0 || !nB0 || !result || !workspace) return fail(SC_EINVAL, "nA0, nB0, result and workspace must be non-NULL");
  if (nsteps < 0) return fail(SC_EINVAL, "nsteps must be >= 0");
  Layout L = layout_of(params);
  if (ws_bytes < L.total) return fail(SC_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
  const int64_t N = (int64_t)params->nx * params->ny * params->nz;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *stage = reinterpret_cast<double *>(static_cast<char *>(workspace) + L.off_fields);
  SC_CUDA(cudaMemcpyAsync(stage, nA0, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  SC_CUDA(cudaMemcpyAsync(stage + N, nB0, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  sc_ctx *c = nullptr;
  st = sc_create(params, stage, stage + N, workspace, ws_bytes, stream, &c);
  if (st != SC_OK) return st;
  st = sc_step(c, nsteps);
  // the 8 results land behind P_in, P_out in the analysis area
  double *res = analysis_pio(c) + 2;
  if (st == SC_OK) st = sc_surface_of_tension(c, SC_PROFILE_RADIAL, centre, bin_width, nbins, 0.0, 0.0, 0.0, res, nullptr);
  if (st == SC_OK) {
    cudaError_t e = cudaMemcpyAsync(result, res, 8 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nA) e = cudaMemcpyAsync(nA, fields_of(c), sizeof(double) * N, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nB) e = cudaMemcpyAsync(nB, fields_of(c) + N, sizeof(double) * N, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = fail(SC_ECUDA, "copying results to the host: %s", cudaGetErrorString(e));
  }
  if (st == SC_OK) st = sc_sync(c);
  sc_destroy(c);
  return st;
}

// ------------------------------------------------------------------ batches
namespace {
constexpr int kGraphSteps = 32;  // steps per graph replay (even: parity preserved)
static_assert(sizeof(unsigned) * (1 + kGraphSteps) <= kAlign, "the batch's counters fit in one aligned slot");

// A batch steps every member with the staged kernel when all of them can take
// it (and none asks for the generic one), else every member with the generic kernel.
bool batch_staged(int32_t n, const sc_params *params) {
  for (int k = 0; k < n; ++k)
    if (!use_staged(&params[k])) return false;
  return true;
}
// Member k's parameters as the batch steps it: the kernel variant of the batch and,
// where the member leaves them to the library, stages and blocks_per_sm resolved
// once for the whole batch from its first member (every member runs in the same launch)
// and the plain tile_z chunking the batch's work list uses.
sc_params member_params(int32_t n, const sc_params *params, int k, bool staged) {
  (void)n;
  sc_params q = params[k];
  q.variant = staged ? 2 : 1;
  sc_params rep = params[0];
  rep.variant = q.variant;
  rep.stages = 0;
  rep.blocks_per_sm = 0;
  const int ty = default_tile_y(&q);
  if (!q.stages) q.stages = effective_stages(&rep, ty);
  if (!q.blocks_per_sm) q.blocks_per_sm = effective_blocks_per_sm(&rep, ty);
  // fixed chunks, the work list is built from them; 64 planes for the staged kernel (the
  // 16-droplet sweep: 3-4 % faster than 32 in every storage)
  if (!q.tile_z) q.tile_z = staged ? (q.nz < 64 ? q.nz : 64) : default_tile_z(&q);
  return q;
}

size_t batch_table_bytes(int32_t n, const sc_params *params, int *nitems_out) {
  const bool staged = batch_staged(n, params);
  int nitems = 0;
  for (int k = 0; k < n; ++k) {
    const sc_params q = member_params(n, params, k, staged);
    const int ty = default_tile_y(&q), tz = default_tile_z(&q);
    nitems += ((q.nx + 31) / 32) * ((q.ny + ty - 1) / ty) * ((q.nz + tz - 1) / tz);
  }
  if (nitems_out) *nitems_out = nitems;
  return align_up(sizeof(StepArgs<double>) * (size_t)n) + align_up(sizeof(int4) * (size_t)nitems) + kAlign;
}

sc_status batch_validate(int32_t n, const sc_params *params) {
  if (n < 1 || n > 4096) return fail(SC_EINVAL, "a batch holds 1 to 4096 lattices");
  if (!params) return fail(SC_EINVAL, "params is NULL");
  for (int k = 0; k < n; ++k) {
    sc_status st = validate(&params[k]);
    if (st != SC_OK) return st;
  }
  const bool staged = batch_staged(n, params);
  const sc_params a = member_params(n, params, 0, staged);
  const int tya = default_tile_y(&a);
  for (int k = 0; k < n; ++k) {
    if (!staged && params[k].variant == 2)
      return fail(SC_EINVAL, "lattice %d asks for the staged kernel, which not every member of the batch can take", k);
    const sc_params b = member_params(n, params, k, staged);
    const int tyb = default_tile_y(&b);
    if (a.lattice != b.lattice || a.stencil != b.stencil || a.storage != b.storage || tya != tyb)
      return fail(SC_EINVAL, "all lattices of a batch share lattice, stencil, storage and tile_y");
    if (staged && (effective_stages(&a, tya) != effective_stages(&b, tyb) ||
                   effective_blocks_per_sm(&a, tya) != effective_blocks_per_sm(&b, tyb)))
      return fail(SC_EINVAL, "all lattices of a batch share stages and blocks_per_sm");
  }
  return SC_OK;
}
}  // namespace

namespace {
// The work list of the members still stepped, (member, x tile, y tile, z chunk) per block,
// uploaded to the batch's item table (synchronously: no launch of the batch is in flight).
sc_status batch_upload_items(sc_batch *b) {
  int total = 0;
  for (int k = 0; k < b->n; ++k) {
    if (b->retired[k]) continue;
    const sc_ctx *c = b->ctx[k];
    total += ((c->p.nx + 31) / 32) * ((c->p.ny + c->tile_y - 1) / c->tile_y) * ((c->p.nz + c->tile_z - 1) / c->tile_z);
  }
  b->nitems = total;
  if (total == 0) return SC_OK;
  int4 *items = new (std::nothrow) int4[total];
  if (!items) return fail(SC_ENOMEM, "host allocation failed");
  int m = 0;
  for (int k = 0; k < b->n; ++k) {
    if (b->retired[k]) continue;
    const sc_ctx *c = b->ctx[k];
    const int gx = (c->p.nx + 31) / 32, gy = (c->p.ny + c->tile_y - 1) / c->tile_y,
              gz = (c->p.nz + c->tile_z - 1) / c->tile_z;
    for (int z = 0; z < gz; ++z)
      for (int y = 0; y < gy; ++y)
        for (int x = 0; x < gx; ++x) items[m++] = make_int4(k, x, y, z);
  }
  cudaError_t e = cudaMemcpyAsync(b->items_dev, items, sizeof(int4) * total, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  delete[] items;
  if (e != cudaSuccess) return fail(SC_ECUDA, "uploading the batch work list: %s", cudaGetErrorString(e));
  return SC_OK;
}

// The persistent form: a graph of two nodes, the barrier and ticket counters zeroed, then one
// cooperative launch of the persistent kernel running kGraphSteps steps from swap 0, with as many
// blocks as there are work items but at most the co-resident blocks of the device.  False (nothing built) when the
// device cannot hold a useful grid.
bool batch_build_persistent(sc_batch *b) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, b->pkernel, 32 * b->tile_y, b->psmem) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    return false;
  }
  b->pgrid = b->nitems < sms * occ ? b->nitems : sms * occ;
  cudaError_t e = cudaGraphCreate(&b->graph, 0);
  cudaGraphNode_t zero = nullptr, node = nullptr;
  if (e == cudaSuccess) {
    cudaMemsetParams mp;
    memset(&mp, 0, sizeof(mp));
    mp.dst = b->counter;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned);
    mp.width = 1 + kGraphSteps;  // the barrier counter and one ticket counter per step
    mp.height = 1;
    e = cudaGraphAddMemsetNode(&zero, b->graph, nullptr, 0, &mp);
  }
  void *argp = b->args_dev;
  void *itemp = b->items_dev;
  int nitems = b->nitems, nsteps = kGraphSteps, swap0 = 0, nlat = b->n;
  unsigned *counter = b->counter;
  void *kp[7] = {&argp, &itemp, &nitems, &nsteps, &swap0, &counter, &nlat};
  if (e == cudaSuccess) {
    cudaKernelNodeParams np;
    memset(&np, 0, sizeof(np));
    np.func = const_cast<void *>(b->pkernel);
    np.gridDim = dim3(b->pgrid);
    np.blockDim = dim3(32, b->tile_y);
    np.sharedMemBytes = (unsigned)b->psmem;
    np.kernelParams = kp;
    e = cudaGraphAddKernelNode(&node, b->graph, &zero, 1, &np);
  }
  if (e == cudaSuccess) {
    cudaLaunchAttributeValue v;
    memset(&v, 0, sizeof(v));
    v.cooperative = 1;
    e = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->pgrid = 0;
    cudaGetLastError();
    return false;
  }
  return true;
}

// A graph of kGraphSteps steps over the current work list, swap = 0, 1, 0, 1, ...: the persistent
// form where the batch has one, else kGraphSteps chained launches (none when no member is left).
sc_status batch_build_graph(sc_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->pgrid = 0;
  if (b->nitems == 0) return SC_OK;
  if (b->pkernel && !b->persist_off && batch_build_persistent(b)) return SC_OK;
  cudaError_t e = cudaGraphCreate(&b->graph, 0);
  cudaGraphNode_t prev = nullptr;
  int swaps[2] = {0, 1};
  void *argp = b->args_dev;
  void *itemp = b->items_dev;
  for (int t = 0; t < kGraphSteps && e == cudaSuccess; ++t) {
    void *kp[3] = {&argp, &itemp, &swaps[t & 1]};
    cudaKernelNodeParams np;
    memset(&np, 0, sizeof(np));
    np.func = const_cast<void *>(b->kernel);
    np.gridDim = dim3(b->nitems);
    np.blockDim = dim3(32, b->tile_y);
    np.sharedMemBytes = (unsigned)b->smem;
    np.kernelParams = kp;
    cudaGraphNode_t node;
    e = cudaGraphAddKernelNode(&node, b->graph, prev ? &prev : nullptr, prev ? 1 : 0, &np);
    prev = node;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return fail(SC_ECUDA, "building the batch graph: %s", cudaGetErrorString(e));
  return SC_OK;
}
}  // namespace

size_t sc_batch_workspace_bytes(int32_t n, const sc_params *params) {
  if (batch_validate(n, params) != SC_OK) return 0;
  size_t total = 0;
  for (int k = 0; k < n; ++k) total += layout_of(&params[k]).total;
  return total + batch_table_bytes(n, params, nullptr);
}

sc_status sc_batch_create(int32_t n, const sc_params *params, const double *const *nA0, const double *const *nB0,
                          void *workspace, size_t ws_bytes, void *stream, sc_batch **out) {
  if (!out) return fail(SC_EINVAL, "out is NULL");
  *out = nullptr;
  sc_status st = batch_validate(n, params);
  if (st != SC_OK) return st;
  if (!nA0 || !nB0 || !workspace) return fail(SC_EINVAL, "initial fields and workspace must be non-NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return fail(SC_EINVAL, "workspace must be 256-byte aligned");
  const size_t need = sc_batch_workspace_bytes(n, params);
  if (ws_bytes < need) return fail(SC_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, need);
  sc_batch *b = new (std::nothrow) sc_batch;
  if (!b) return fail(SC_ENOMEM, "host allocation failed");
  memset(b, 0, sizeof(*b));
  b->n = n;
  b->stream = static_cast<cudaStream_t>(stream);
  b->ctx = new (std::nothrow) sc_ctx *[n];
  if (!b->ctx) {
    delete b;
    return fail(SC_ENOMEM, "host allocation failed");
  }
  for (int k = 0; k < n; ++k) b->ctx[k] = nullptr;
  char *ws = static_cast<char *>(workspace);
  size_t off = 0;
  const bool staged = batch_staged(n, params);
  for (int k = 0; k < n; ++k) {
    sc_params pk = member_params(n, params, k, staged);
    const size_t bytes = layout_of(&pk).total;
    st = sc_create(&pk, nA0[k], nB0[k], ws + off, bytes, stream, &b->ctx[k]);
    if (st != SC_OK) {
      sc_batch_destroy(b);
      return st;
    }
    b->ctx[k]->in_batch = 1;
    off += bytes;
  }
  // tables: per-lattice arguments (parity 0) and the block work list
  int nitems = 0;
  batch_table_bytes(n, params, &nitems);
  b->nitems = nitems;
  b->tile_y = b->ctx[0]->tile_y;
  b->args_dev = ws + off;
  off += align_up(sizeof(StepArgs<double>) * (size_t)n);
  b->items_dev = reinterpret_cast<int4 *>(ws + off);
  off += align_up(sizeof(int4) * (size_t)nitems);
  b->counter = reinterpret_cast<unsigned *>(ws + off);
  const int storage = params[0].storage;
  const size_t arg_size = storage == SC_STORE_F64 ? sizeof(StepArgs<double>) : sizeof(StepArgs<float>);
  std::string host_args(arg_size * n, '\0');
  for (int k = 0; k < n; ++k) {
    sc_ctx *c = b->ctx[k];
    if (storage == SC_STORE_F64) {
      StepArgs<double> a = step_args<double>(c);
      memcpy(&host_args[arg_size * k], &a, arg_size);
    } else {
      StepArgs<float> a = step_args<float>(c);
      memcpy(&host_args[arg_size * k], &a, arg_size);
    }
  }
  cudaError_t e = cudaMemcpyAsync(b->args_dev, host_args.data(), arg_size * n, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    sc_batch_destroy(b);
    return fail(SC_ECUDA, "uploading batch tables: %s", cudaGetErrorString(e));
  }
  b->retired = new (std::nothrow) char[n];
  if (!b->retired) {
    sc_batch_destroy(b);
    return fail(SC_ENOMEM, "host allocation failed");
  }
  memset(b->retired, 0, n);
  b->active = n;
  st = batch_upload_items(b);
  if (st != SC_OK) {
    sc_batch_destroy(b);
    return st;
  }
  if (b->nitems != nitems) {
    sc_batch_destroy(b);
    return fail(SC_EINVAL, "batch work list size mismatch (%d vs %d)", b->nitems, nitems);
  }
  const int lat = params[0].lattice == SC_D3Q19 ? kD3Q19 : kD2Q9;
  const int sten = params[0].stencil == SC_FORCE_E6 ? kE6 : kE4;
  b->staged = staged ? 1 : 0;
  bool all_t1 = true;  // every member has tau_A = tau_B = 1: the momentum-carry instantiation
  for (int k = 0; k < n; ++k) all_t1 = all_t1 && tau_one(&params[k]);
  if (staged) {
    const int ns = b->ctx[0]->stages, mb = b->ctx[0]->blocks_per_sm;
    bool any_self = false;
    for (int k = 0; k < n; ++k) any_self = any_self || has_self(&params[k]);
    switch (storage) {
      case SC_STORE_F32: b->kernel = batched_staged_kernel_f32(b->tile_y, ns, mb, any_self, all_t1, &b->smem); break;
      case SC_STORE_F16: b->kernel = batched_staged_kernel_f16(b->tile_y, ns, mb, any_self, all_t1, &b->smem); break;
      case SC_STORE_BF16: b->kernel = batched_staged_kernel_bf16(b->tile_y, ns, mb, any_self, all_t1, &b->smem); break;
      default: b->kernel = batched_staged_kernel_f64(b->tile_y, ns, mb, any_self, all_t1, &b->smem); break;
    }
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop) {
      switch (storage) {
        case SC_STORE_F32: b->pkernel = persistent_staged_kernel_f32(b->tile_y, ns, mb, any_self, all_t1, &b->psmem); break;
        case SC_STORE_F16: b->pkernel = persistent_staged_kernel_f16(b->tile_y, ns, mb, any_self, all_t1, &b->psmem); break;
        case SC_STORE_BF16: b->pkernel = persistent_staged_kernel_bf16(b->tile_y, ns, mb, any_self, all_t1, &b->psmem); break;
        default: b->pkernel = persistent_staged_kernel_f64(b->tile_y, ns, mb, any_self, all_t1, &b->psmem); break;
      }
    }
    cudaGetLastError();  // a configuration without a persistent form leaves the per-step launches
  } else {
    switch (storage) {
      case SC_STORE_F32: b->kernel = batched_kernel_f32(lat, sten, b->tile_y, all_t1, &b->smem); break;
      case SC_STORE_F16: b->kernel = batched_kernel_f16(lat, sten, b->tile_y, all_t1, &b->smem); break;
      case SC_STORE_BF16: b->kernel = batched_kernel_bf16(lat, sten, b->tile_y, all_t1, &b->smem); break;
      default: b->kernel = batched_kernel_f64(lat, sten, b->tile_y, all_t1, &b->smem); break;
    }
  }
  if (!b->kernel) {
    sc_batch_destroy(b);
    return fail(SC_EUNSUPPORTED, "no batched kernel for this lattice / stencil / tile_y / stages / blocks_per_sm");
  }
  st = batch_build_graph(b);
  if (st != SC_OK) {
    sc_batch_destroy(b);
    return st;
  }
  *out = b;
  return SC_OK;
}

sc_status sc_batch_step(sc_batch *b, int64_t nsteps) {
  if (!b) return fail(SC_EINVAL, "batch is NULL");
  if (nsteps < 0) return fail(SC_EINVAL, "nsteps must be >= 0");
  if (b->nitems == 0) return SC_OK;  // every member retired
  auto single = [&]() -> cudaError_t {
    void *argp = b->args_dev;
    void *itemp = b->items_dev;
    int swap = (int)(b->steps & 1);
    void *kp[3] = {&argp, &itemp, &swap};
    cudaError_t e = cudaLaunchKernel(b->kernel, dim3(b->nitems), dim3(32, b->tile_y), kp, b->smem, b->stream);
    b->steps++;
    b->launches++;
    return e;
  };
  while (nsteps > 0) {
    cudaError_t e;
    if ((b->steps & 1) == 0 && nsteps >= kGraphSteps) {
      e = cudaGraphLaunch(b->exec, b->stream);
      b->steps += kGraphSteps;
      b->launches += kGraphSteps;
      nsteps -= kGraphSteps;
    } else {
      e = single();
      nsteps -= 1;
    }
    if (e != cudaSuccess) return fail(SC_ECUDA, "batched step: %s", cudaGetErrorString(e));
  }
  for (int k = 0; k < b->n; ++k) {
    if (b->retired[k]) continue;
    b->ctx[k]->cur = (int)(b->steps & 1);
    b->ctx[k]->steps = b->steps;
    b->ctx[k]->launches = b->launches;
  }
  return SC_OK;
}

sc_status sc_batch_retire(sc_batch *b, int32_t k) {
  if (!b) return fail(SC_EINVAL, "batch is NULL");
  if (k < 0 || k >= b->n) return fail(SC_EINVAL, "no batch member %d", k);
  if (b->retired[k]) return SC_OK;
  SC_CUDA(cudaStreamSynchronize(b->stream));
  b->retired[k] = 1;
  b->active -= 1;
  sc_status st = batch_upload_items(b);
  if (st == SC_OK) st = batch_build_graph(b);
  return st;
}

int32_t sc_batch_active(const sc_batch *b) { return b ? b->active : 0; }

sc_status sc_batch_set_persistent(sc_batch *b, int32_t on) {
  if (!b) return fail(SC_EINVAL, "batch is NULL");
  if (on != 0 && on != 1) return fail(SC_EINVAL, "on must be 0 or 1");
  if (on && !b->pkernel) return fail(SC_EUNSUPPORTED, "the batch has no persistent form (generic kernel or no cooperative launch)");
  SC_CUDA(cudaStreamSynchronize(b->stream));
  b->persist_off = !on;
  sc_status st = batch_build_graph(b);
  if (st == SC_OK && on && b->nitems > 0 && b->pgrid == 0)
    return fail(SC_EUNSUPPORTED, "the persistent launch could not be built on this device");
  return st;
}

sc_ctx *sc_batch_member(sc_batch *b, int32_t k) {
  if (!b || k < 0 || k >= b->n) {
    fail(SC_EINVAL, "no such batch member");
    return nullptr;
  }
  return b->ctx[k];
}

int64_t sc_batch_launches(const sc_batch *b) { return b ? b->launches : 0; }
int32_t sc_batch_variant(const sc_batch *b) { return b ? (b->staged ? (b->pgrid > 0 ? 3 : 2) : 1) : 0; }

void sc_batch_destroy(sc_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ctx)
    for (int k = 0; k < b->n; ++k) delete b->ctx[k];
  delete[] b->ctx;
  delete[] b->retired;
  delete b;
}

sc_status sc_step_config(const sc_ctx *c, int32_t *out, int32_t n) {
  if (!c || !out) return fail(SC_EINVAL, "ctx and out must be non-NULL");
  if (n < 8) return fail(SC_EINVAL, "out must hold 8 values, got room for %d", n);
  const int64_t grid = c->zbal_k > 0 ? (int64_t)c->zbal_k * c->zbal_cols + c->zbal_rem
                                     : (int64_t)((c->p.nx + 31) / 32) * ((c->p.ny + c->tile_y - 1) / c->tile_y) *
                                           ((c->p.nz + c->tile_z - 1) / c->tile_z);
  const int32_t v[8] = {c->staged ? 2 : 1, c->tile_y, c->tile_z, c->staged ? c->stages : 0,
                        c->staged ? c->blocks_per_sm : 0, (int32_t)grid, c->zbal_k, c->zbal_rem};
  for (int k = 0; k < 8; ++k) out[k] = v[k];
  return SC_OK;
}

int64_t sc_kernel_launches(const sc_ctx *c) { return c ? c->launches : 0; }

sc_status sc_reference_density(const sc_ctx *c, double nbar[2]) {
  if (!c || !nbar) return fail(SC_EINVAL, "ctx and nbar must be non-NULL");
  nbar[0] = c->nbar[0];
  nbar[1] = c->nbar[1];
  return SC_OK;
}

void sc_destroy(sc_ctx *c) {
  if (!c) return;
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

const char *sc_last_error(void) { return g_err.c_str(); }

}  // extern "C"
