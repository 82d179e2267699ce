/*
 * sc.h -- C ABI of a GB300 (sm_103a) library for the two-component Shan-Chen
 * lattice Boltzmann method and the surface-of-tension analysis of
 * Lulli et al., "Mesoscale Modelling of the Tolman Length in Multi-component
 * Systems" (arXiv:2112.02574).
 *
 * Conventions for every entry point
 *   - Return value: sc_status.  Nothing here aborts, exits or throws.  On an
 *     error the entry point returns before launching any work, and
 *     sc_last_error() describes the failure (a per-thread message).
 *   - Memory: the caller owns every buffer (inputs, outputs, workspace).  A
 *     pointer documented as "device" must be CUDA device memory on the current
 *     device, "host" must be host memory (pinned or pageable).  The library
 *     allocates no device memory except where an entry point says so; its
 *     context (sc_ctx) is a small host object holding offsets into the caller's
 *     workspace.
 *   - Streams: all device work of a context is issued on the stream given to
 *     sc_create (a cudaStream_t passed as void*; NULL = legacy default stream)
 *     and is asynchronous unless the entry point says it synchronises.
 *   - Lattice fields are [nz][ny][nx] with x fastest; site s = x + nx*(y + ny*z);
 *     every direction is periodic.
 *   - Populations in the "natural" FP64 layout are f[J][i][s], J = 0 (A), 1 (B),
 *     i in the velocity order below, and hold the pre-collision populations
 *     f_i^J(x, t) of Eq. lbm.
 *   - Units are lattice units; c_s^2 = 1/3 (section 2 and section 4).
 *
 * Velocity order (opposite directions adjacent):
 *   D3Q19: 0 (0,0,0); 1..6 (+x)(-x)(+y)(-y)(+z)(-z);
 *          7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1)
 *          13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 *   D2Q9:  0 (0,0); 1..4 (+x)(-x)(+y)(-y); 5 (1,1) 6 (-1,-1) 7 (1,-1) 8 (-1,1)
 */
#ifndef SC_H
#define SC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SC_OK = 0,
  SC_EINVAL = 1,        /* bad argument (null pointer, size, parameter out of range) */
  SC_ENOMEM = 2,        /* workspace smaller than sc_workspace_bytes() */
  SC_ECUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  SC_ENAN = 4,          /* a step met a non-finite density, or a non-positive one while
                           psi = exp(-1/n) is in use (with psi = n the method stays defined
                           for transiently negative densities, and they are not flagged) */
  SC_ETIMEOUT = 5,      /* a bounded device-side wait ran out */
  SC_EUNSUPPORTED = 6   /* valid request the library has no kernel for */
} sc_status;

typedef enum { SC_D2Q9 = 0, SC_D3Q19 = 1 } sc_lattice;
/* Forcing stencil of Eq. sc_force: E4 = the velocity set's own non-rest vectors
 * with W(1) = 1/6, W(2) = 1/12 (section 2; D2Q9: 1/3, 1/12); E6 = all integer
 * vectors with |xi|^2 = 1..4 and W = 2/15, 1/15, 1/60, 1/120 (D3Q19 only). */
typedef enum { SC_FORCE_E4 = 0, SC_FORCE_E6 = 1 } sc_stencil;
/* Pseudopotential of the self-coupling term: psi = n, or psi = exp(-1/n) (section 4). */
typedef enum { SC_PSI_N = 0, SC_PSI_EXP = 1 } sc_psi;
/* Population storage.  F32/F64 store deviations g_i = f_i - w_i nbar_J from a
 * rest equilibrium with the mean initial density nbar_J.  F16/BF16 store the
 * deviation from each site's own rest equilibrium, (f*_i(s) - w_i n_J(s)) 2^k(J)
 * (F16: a power-of-two scale per component fixed at sc_create; BF16: unscaled),
 * with n_J(s) the site's density when it was written (the sum of the values
 * stored at s) and n_J(s) - nbar_J kept beside them as an FP32 pair per site.
 * Collision arithmetic is FP32 for F32/F16/BF16 and FP64 for F64.  In device memory the two components of a
 * direction and site are adjacent ([i][site][J]); sc_get_state / sc_set_state
 * copy that buffer followed, for F16/BF16, by the [site][J] FP32 density
 * deviations. */
typedef enum { SC_STORE_F32 = 0, SC_STORE_F16 = 1, SC_STORE_BF16 = 2, SC_STORE_F64 = 3 } sc_storage;
typedef enum { SC_PROFILE_RADIAL = 0, SC_PROFILE_PLANAR_Z = 1, SC_PROFILE_AXIS_X = 2 } sc_profile_kind;

/* Model and layout parameters.  Couplings follow Eq. sc_force literally:
 * F_A = -G c_s^2 n_A sum_a W n_B(x+xi_a) xi_a - G_AA c_s^2 psi_A sum_a W psi_A(x+xi_a) xi_a. */
typedef struct {
  int32_t nx, ny, nz;  /* lattice size, each >= 1; nz == 1 for D2Q9 */
  int32_t lattice;     /* sc_lattice */
  int32_t stencil;     /* sc_stencil */
  int32_t psi_self;    /* sc_psi */
  int32_t storage;     /* sc_storage */
  int32_t tile_y;      /* step-kernel tile rows (1, 2, 4 or 8; 16 staged only); 0 = library default */
  int32_t tile_z;      /* planes per step-kernel work item (>= 1); 0 = library default
                          (D3Q19: staged kernel 128 or 64 planes where that grid fills
                          eight waves of the GPU; either kernel 32 where that fills four,
                          else a balanced split whose grid fills whole waves; a batch: 64
                          staged, 32 generic; D2Q9: 1) */
  int32_t variant;     /* step kernel: 0 = automatic (staged where it can run), 1 = generic
                          (any size, any stencil), 2 = cp.async-staged (D3Q19, E4, nx >= 32
                          a multiple of the sites per 16-byte chunk: 1 F64, 2 F32, 4 F16 and
                          BF16; tile_y 4, 8 or 16, F64 tile_y 4 only); both kernels compute
                          the same numbers */
  int32_t stages;      /* staged kernel copy pipeline: 1 or 2 planes in flight; 0 = default */
  int32_t blocks_per_sm; /* staged kernel register budget: resident blocks per SM it must allow
                          (tile_y 4: 2 or 3; tile_y 8: 1 or 2; tile_y 16: 1); 0 = default.  stages and
                          blocks_per_sm change speed only, never the numbers */
  double tau[2];       /* tau_A, tau_B > 1/2 (Eq. omega_i) */
  double G;            /* inter-component coupling G */
  double G_self[2];    /* self couplings G_AA, G_BB */
} sc_params;

typedef struct sc_ctx sc_ctx;

/* Bytes of device workspace sc_create needs for these parameters (0 if the
 * parameters are invalid).  Layout: two population buffers, FP64 field planes
 * for the analysis kernels, reduction scratch and a status word. */
size_t sc_workspace_bytes(const sc_params *params);

/* Create a simulation (section 2; initial state of section 4: rest equilibrium
 * f_i = w_i n_J with u = 0).  nA0, nB0: device FP64 [N] initial densities
 * (each > 0).  workspace: device memory of ws_bytes >= sc_workspace_bytes(),
 * 256-byte aligned, owned by the caller and kept alive until sc_destroy.
 * Enqueues the initialisation on `stream` and synchronises it. */
sc_status sc_create(const sc_params *params, const double *nA0, const double *nB0, void *workspace,
                    size_t ws_bytes, void *stream, sc_ctx **out);

/* Advance nsteps >= 0 time steps of Eq. lbm (BGK of Eq. omega_i, Guo forcing,
 * equilibrium of Eq. feq, common velocity of Eq. u, force of Eq. sc_force,
 * streaming).  One fused kernel launch per step; asynchronous.  Runs of 32 steps
 * are replayed from a CUDA graph of 32 launches that the context captures once,
 * on a private stream, the first time such a run comes up (the replay goes to the
 * context's stream; if the capture is not possible the steps are plain launches). */
sc_status sc_step(sc_ctx *ctx, int64_t nsteps);

/* Densities n_A, n_B (device FP64 [N] each) and, if u != NULL, the common
 * velocity of Eq. u (device FP64 [3][N], force included).  Asynchronous. */
sc_status sc_moments(sc_ctx *ctx, double *nA, double *nB, double *u);

/* Pre-collision populations in the natural FP64 layout (device [2][Q][N]). */
sc_status sc_get_populations(sc_ctx *ctx, double *f);
/* Replace the state by natural-layout FP64 populations (device [2][Q][N]);
 * values are rounded to the storage format. */
sc_status sc_set_populations(sc_ctx *ctx, const double *f);

/* Raw state (checkpoint / resume, bit-exact): bytes == sc_state_bytes(ctx);
 * dst / src are device memory. */
size_t sc_state_bytes(const sc_ctx *ctx);
sc_status sc_get_state(sc_ctx *ctx, void *dst, size_t bytes);
sc_status sc_set_state(sc_ctx *ctx, const void *src, size_t bytes);

/* Pressure-tensor profile (Eq. sm:pt, accumulated in FP64).  out: device FP64
 * [nbins][6] rows (coordinate, P_N, P_T, n_A, n_B, count), means per bin,
 * empty bins all zero.
 *   RADIAL:   shells of width bin_width around centre (minimum image), P_N =
 *             rhat.P.rhat, P_T = (tr P - P_N)/(d - 1), at r = 0 both tr P/d
 *             (decomposition of Eq. pt_projection, section 3);
 *   PLANAR_Z: one bin per plane z < nbins, P_N = <P^zz>, P_T = <(P^xx+P^yy)/2>
 *             (flat interface, section 4);
 *   AXIS_X:   sites (cx + k, cy, cz), k < nbins <= nx (larger nbins is
 *             SC_EINVAL: each row holds exactly one site), P_N = P^xx, P_T = P^yy
 *             (section 3, the paper's own estimator).
 * Deterministic: per-block partial sums in a fixed order.  Asynchronous. */
sc_status sc_pressure_profile(sc_ctx *ctx, int32_t kind, const double centre[3], double bin_width, int32_t nbins,
                              double *out);

/* Bulk pressure of Eq. bulkp at one node; out: device FP64 [1].  Asynchronous. */
sc_status sc_bulk_pressure_at(sc_ctx *ctx, const int32_t node[3], double *out);

/* Generalized surface tension minimum from a profile (section 3, Eqs.
 * gen_sigma, gen_d_sigma), in FP64 on the device.  rows: device FP64
 * [nbins][6] as written by sc_pressure_profile; P_in_out: device FP64 [2].
 * Integrals run over the non-empty rows up to the last one (r_max): the
 * pressure-jump part exactly, P_T by the trapezoid rule, so that
 * sigma[R] = dP R/3 + C/R^2 (dim 3) or dP R/2 + C/R (dim 2) with
 * C = int_0^r_max r^(dim-1) (P_out - P_T) dr.  out: device FP64 [8] =
 * (dP, C, R_s, sigma_s, R_grid, sigma_grid, P_in, P_out) where R_s is the
 * closed-form minimum, sigma_s = dP R_s / 2 (dim 3) or dP R_s (dim 2), and
 * (R_grid, sigma_grid) the parabolic interpolation of the minimum of sigma[R]
 * sampled on [R_lo, R_hi] with step R_step (the paper's procedure).
 * stream: cudaStream_t as void*.  Asynchronous. */
sc_status sc_sigma_minimum(const double *rows, int32_t nbins, const double *P_in_out, int32_t dim, double R_lo,
                           double R_hi, double R_step, double *out, void *stream);

/* The surface of tension of a droplet in one call: the pressure-tensor profile
 * (as sc_pressure_profile), the bulk pressures of Eq. bulkp at the centre node
 * (P_in) and at the far corner (nx-1, ny-1, nz-1) (P_out, section 4), and the
 * minimum of the generalized surface tension sigma[R] (section 3, Eqs.
 * gen_sigma and gen_d_sigma), all on the device.
 *   kind:      SC_PROFILE_RADIAL (shells of bin_width around centre) or
 *              SC_PROFILE_AXIS_X (the paper's line through the centre node,
 *              unit spacing; bin_width is ignored); anything else is SC_EINVAL.
 *   centre:    host [3] (x, y, z), or NULL for the centre node (nx/2, ny/2, nz/2);
 *              the node nearest to it (periodic) gives P_in.
 *   nbins:     rows of the profile (<= 4096; <= nx for the axis), or 0 for the
 *              largest sphere inside the box (min(nx, ny, nz) / 2 / bin_width; the
 *              axis: nx / 2 rows).
 *   R_lo, R_hi, R_step: grid of the paper's interpolated minimum; 0 picks the
 *              default for each (R_step 0.01, R_lo = R_step, R_hi = nbins x spacing).
 *   out:       device FP64 [8] = (dP, C, R_s, sigma_s, R_grid, sigma_grid, P_in,
 *              P_out), as sc_sigma_minimum.
 *   rows:      device FP64 [nbins][6] that receives the profile, or NULL to keep
 *              it in the context's workspace.
 * Deterministic; asynchronous on the context's stream. */
sc_status sc_surface_of_tension(sc_ctx *ctx, int32_t kind, const double centre[3], double bin_width, int32_t nbins,
                                double R_lo, double R_hi, double R_step, double *out, double *rows);

/* Run diagnostics of sections 2 and 4 in one call, deterministic FP64:
 * out: device FP64 [10] = (mass_A, mass_B, momentum x, y, z (as sc_totals),
 * dU (as sc_velocity_change: u_prev is read and then overwritten with u; NaN
 * when u_prev is NULL), X, Y, Z, W (centre of mass of component `component`
 * over `background`, as sc_centre_of_mass; all NaN when component is -1)).
 * u_prev: device FP64 [3][N] or NULL; component: -1, 0 (A) or 1 (B).
 * Asynchronous on the context's stream. */
sc_status sc_diagnostics(sc_ctx *ctx, double *u_prev, int32_t component, double background, double *out);

/* Convergence measure of section 4 on the velocity field: dU = (1 / N) sum over
 * the sites x of sum_alpha |u_alpha(x) - u_prev_alpha(x)|, with u the common
 * velocity of Eq. u (force included) of the current state; u_prev is then
 * overwritten with u, ready for the next interval.  u_prev: device FP64 [3][N]
 * (e.g. from sc_moments at the start of the interval); out: device FP64 [1].
 * Deterministic; asynchronous on the context's stream. */
sc_status sc_velocity_change(sc_ctx *ctx, double *u_prev, double *out);

/* Centre of mass of component `component` (0: A, 1: B) counted as its density
 * excess over `background`: w(x) = n_J(x) - background, out = (sum w x / W,
 * sum w y / W, sum w z / W, W) in lattice coordinates (no periodic unwrapping:
 * for a droplet away from the box faces, the acceptance test of section 4
 * compares this with the centre node).  out: device FP64 [4].  Deterministic;
 * asynchronous on the context's stream. */
sc_status sc_centre_of_mass(sc_ctx *ctx, int32_t component, double background, double *out);

/* Flat-interface surface tension (section 4, the sigma_0 of Eq. sigma_c):
 * sigma_0 = sum over the planes z >= nbins / 2 of P_N(z) - P_T(z), from the rows
 * of a PLANAR_Z profile (one bin per plane) of a periodic slab whose second
 * interface lies in the upper half.  rows: device FP64 [nbins][6]; out: device
 * FP64 [1].  Deterministic; asynchronous on stream. */
sc_status sc_sigma0_flat(const double *rows, int32_t nbins, double *out, void *stream);

/* Curvature expansion of the surface tension (Eq. sigma_c, section 1; the
 * Tolman length delta and the rigidity combination 2 kbar + k): least squares
 * of sigma_s = sigma_0 (1 - 2 delta / R_s + (2 kbar + k) / R_s^2) over n droplets,
 * in FP64 on the device.  Rs, sigma_s: device FP64 [n], R_s signed (negative for
 * droplets of the other component, section 4); order 1 or 2 (1: no 1/R_s^2
 * term); sigma0: device FP64 [1] holding a fixed sigma_0 (e.g. from
 * sc_sigma0_flat), or NULL to fit it.  out: device FP64 [4] = (sigma_0, delta,
 * 2 kbar + k (NaN for order 1), rms residual of sigma_s).  Needs n >= number of
 * unknowns (order, plus one when sigma_0 is fitted).  Asynchronous on stream. */
sc_status sc_curvature_fit(const double *Rs, const double *sigma_s, int32_t n, int32_t order, const double *sigma0,
                           double *out, void *stream);

/* Pressure-tensor profile without any device allocation.  The paper has no
 * counterpart to this entry point; it exists for callers that cannot allocate
 * device memory at the point of the call -- for instance code that has handed
 * all device memory to its own pool allocator, or that runs where the implicit
 * device synchronisation of cudaMalloc / cudaFree is not allowed.  It computes
 * the same rows as sc_pressure_profile (same kinds, same layout of out), but
 * from caller-provided density fields nA, nB (device FP64 [N], N from params;
 * params gives the lattice, stencil, psi_self, G and G_self) with the
 * pseudopotential evaluated on the fly, and without a context or workspace.
 * Its only scratch is a fixed 4 MiB __device__ array inside this library, which
 * every GPU that loads the library holds until the process exits; nbins may be
 * at most 4096 (larger requests return SC_EINVAL), and at most nx for the x
 * axis.  params must pass the model checks of sc_create (size, lattice,
 * stencil, psi_self, finite couplings).  It calls no cudaMalloc, cudaFree or
 * other allocating routine.  Every call made while its stream is not capturing
 * looks up the array's device address on the current device (a device reset
 * reloads the library's module and may move the array); a call made while the
 * stream captures a CUDA graph reuses the address the last such lookup on that
 * device found, so make the first call on a device, and the first after a
 * device reset, before any stream capture.  All calls share the array and
 * each call overwrites every entry it later reads, so nothing needs clearing;
 * calls that overlap on the GPU (other streams, other host threads) race on
 * it.  out: device FP64 [nbins][6].  stream: cudaStream_t as void*.
 * Asynchronous. */
sc_status sc_pressure_profile_noalloc(const sc_params *params, const double *nA, const double *nB, int32_t kind,
                                      const double centre[3], double bin_width, int32_t nbins, double *out,
                                      void *stream);

/* Conserved totals, FP64, deterministic: out device [5] = (mass_A, mass_B,
 * momentum x, y, z) summed over the lattice (section 2).  Asynchronous. */
sc_status sc_totals(sc_ctx *ctx, double *out);

/* Wait for the context's stream and report device-side errors (SC_ENAN, or
 * SC_ETIMEOUT for a bounded wait that ran out; see sc_status; the flag is then
 * cleared). */
sc_status sc_sync(sc_ctx *ctx);

/* Self-test of the bounded device-side wait that a persistent batch launch
 * uses between time steps: one block on ctx's stream waits at that grid barrier
 * for an arrival that never comes; after max_polls polls (1 <= max_polls <=
 * 2^20; polls back off from 64 ns to 4 us) the wait runs out and sets the
 * timeout bit of ctx's status word, so that the next sc_sync returns
 * SC_ETIMEOUT and clears it.  The context's state is untouched and it stays
 * usable.  Asynchronous; SC_EINVAL for a NULL ctx or max_polls out of range. */
sc_status sc_selftest_wait_timeout(sc_ctx *ctx, int32_t max_polls);

/* Convenience entry point with HOST buffers: create, run nsteps and read the
 * densities back.  nA0, nB0: host FP64 [N] in; nA, nB: host FP64 [N] out.
 * The workspace is device memory as for sc_create.  Synchronous. */
sc_status sc_run_host(const sc_params *params, const double *nA0, const double *nB0, int64_t nsteps, double *nA,
                      double *nB, void *workspace, size_t ws_bytes, void *stream);

/* The method's result with HOST buffers in and out: create from host initial
 * densities, run nsteps, then sc_surface_of_tension with a radial profile
 * (centre, bin_width, nbins as there; the default R grid) and read the results
 * back.  nA0, nB0: host FP64 [N]; nA, nB: host FP64 [N] receiving the final
 * densities, or NULL to skip that copy; result: host FP64 [8] as the out of
 * sc_surface_of_tension.  The workspace is device memory as for sc_create.
 * Synchronous. */
sc_status sc_run_host_sigma(const sc_params *params, const double *nA0, const double *nB0, int64_t nsteps,
                           const double centre[3], double bin_width, int32_t nbins, double *nA, double *nB,
                           double *result, void *workspace, size_t ws_bytes, void *stream);

/* ---- batches: several lattices stepped together ----
 * The batched radius sweep: lattices of different sizes and parameters (same
 * lattice type, stencil, storage and tile_y) stepped together over a work list
 * of (lattice, tile) items, from a CUDA graph (built explicitly, no stream
 * capture).  The kernel is the staged one when every member can take it
 * (variant 0 or 2, D3Q19, E4, nx >= 32 a multiple of the chunk sites; members
 * then share stages and blocks_per_sm), else the generic one; a member with
 * variant 2 in a batch that cannot be staged is an error (SC_EINVAL).
 * By default (where the device has cooperative launch; see
 * sc_batch_set_persistent) a staged batch runs 32 time steps of every member in
 * ONE persistent cooperative launch: in each step its blocks draw the work
 * items from a ticket counter, then meet at a grid-wide barrier before the
 * next; a barrier wait that runs out (2^20 polls, a few seconds) sets bit 1 of
 * every member's status word, reported by sc_sync as SC_ETIMEOUT.  Otherwise,
 * and for a generic batch, the graph replays 32 chained launches, one per step.  Steps outside whole runs of
 * 32 are single launches.  Each member is an ordinary context for the analysis
 * entry points (sc_moments, sc_pressure_profile, sc_bulk_pressure_at, ...);
 * sc_step refuses batch members. */
typedef struct sc_batch sc_batch;
/* Device workspace for n lattices (0 if the parameters are invalid). */
size_t sc_batch_workspace_bytes(int32_t n, const sc_params *params);
/* params[n]; nA0[k], nB0[k]: device FP64 [N_k] initial densities of lattice k.
 * Synchronises the stream once (initialisation and table upload). */
sc_status sc_batch_create(int32_t n, const sc_params *params, const double *const *nA0, const double *const *nB0,
                          void *workspace, size_t ws_bytes, void *stream, sc_batch **out);
/* Advance every member by nsteps time steps (section 2); asynchronous. */
sc_status sc_batch_step(sc_batch *batch, int64_t nsteps);
/* Choose how whole runs of 32 steps of a staged batch go out: on = 1 (the
 * default where the device has cooperative launch) one persistent launch per
 * run, on = 0 one launch per step.  Both forms give the same members bit for
 * bit.  Waits for the batch's stream.  SC_EUNSUPPORTED for on = 1 when the
 * batch has no persistent form (a generic batch, or no cooperative launch). */
sc_status sc_batch_set_persistent(sc_batch *batch, int32_t on);
/* Member k as a context (owned by the batch; NULL if k is out of range). */
sc_ctx *sc_batch_member(sc_batch *batch, int32_t k);
/* Time steps issued to every member so far (a persistent launch counts once
 * per step it runs). */
int64_t sc_batch_launches(const sc_batch *batch);
/* Step kernel of the batch: 1 generic, 2 staged (one launch per step), 3 staged
 * and persistent (0 for NULL). */
int32_t sc_batch_variant(const sc_batch *batch);
/* Stop stepping member k (section 4 runs each droplet until it has converged,
 * so members of a sweep finish at different times).  The member keeps its state
 * and step count and stays usable for the analysis entry points; later
 * sc_batch_step calls launch over the remaining members only (work list and
 * graph rebuilt here).  Retiring a retired member does nothing.  Synchronises
 * the batch's stream. */
sc_status sc_batch_retire(sc_batch *batch, int32_t k);
/* Members still stepped (not retired). */
int32_t sc_batch_active(const sc_batch *batch);
void sc_batch_destroy(sc_batch *batch);

/* The step kernel this context launches: out[0..8) = variant (1 generic, 2
 * staged), tile_y, tile_z, stages, blocks_per_sm, blocks per launch, balanced
 * split K (0: plain grid of tile_z chunks), columns with K + 1 chunks.  n: room
 * in out (>= 8).  Host only, no synchronisation. */
sc_status sc_step_config(const sc_ctx *ctx, int32_t *out, int32_t n);

/* Number of step-kernel launches issued by this context so far. */
int64_t sc_kernel_launches(const sc_ctx *ctx);

/* Mean initial densities nbar_J used as the storage reference (host out [2]). */
sc_status sc_reference_density(const sc_ctx *ctx, double nbar[2]);

/* Release the context (host memory only; the workspace stays the caller's). */
void sc_destroy(sc_ctx *ctx);

/* Last error message of the calling thread ("" if none). */
const char *sc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SC_H */
