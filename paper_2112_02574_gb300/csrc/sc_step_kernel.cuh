// The fused two-component Shan-Chen time step (arXiv:2112.02574, section 2).
//
// One launch = one time step of Eq. lbm for both components:
//   pull-streaming  f_i(x, t) = f*_i(x - xi_i, t - 1)
//   moments         n_J = sum_i f_i, j_J = sum_i f_i xi_i
//   pseudopotential psi_J = exp(-1/n_J) or n_J
//   force           Eq. sc_force (cross term on n, self term on psi)
//   velocity        n u = sum_J (j_J + F_J / 2)                      (Eq. u)
//   BGK + Guo       f* = f - (f - f^eq)/tau_J + (1 - 1/(2 tau_J)) F_i (Eqs. omega_i, Guo, feq)
// The state kept in memory is f* at the collision site, so the next step
// pulls again; populations are stored as deviations g = f - w_i nbar_J, both
// components of a direction and site side by side, and every quantity that
// exists per component is computed as an (A, B) pair.
//
// Blocking (the force at x needs n at x + xi_a for the same time level, and
// those come from other sites' streamed populations): a block owns a column
// chunk of 32 x TY sites in x-y and tile_z planes in z, and marches along z.
// For every plane it recomputes the density (and psi) deviations of the tile
// plus a halo of HALO sites into a ring of shared-memory planes; once planes
// c - HALO .. c + HALO are in the ring it collides plane c.  The halo sums
// re-read neighbouring sites' populations, which the neighbouring blocks read
// at about the same time (L2 hits); every population of the domain is read
// from HBM once and written once per step.  No block waits on another block.
#pragma once

#include "sc_common.cuh"

namespace scgb {

// Weight w_i of direction i as a component pair, in the step's units (scaled_units).
template <int LAT, class ST, class CT>
__device__ __forceinline__ P2<CT> wpair(int i, P2<CT> scale) {
  if constexpr (scaled_units<ST>()) return pmul(pbc(CT(Lattice<LAT>::w(i))), scale);
  return pbc(CT(Lattice<LAT>::w(i)));
}
// A sum of pairs in the step's units, as a natural value.
template <class ST, class CT>
__device__ __forceinline__ P2<CT> unscale(P2<CT> v, P2<CT> inv_scale) {
  if constexpr (scaled_units<ST>()) return pmul(v, inv_scale);
  return v;
}

// Pull the Q population pairs arriving at site (gx, gy, gz) and return their
// sum (the density deviations, natural units); values go to v[] (step units) when
// V is true.  Values are deviations from w_i nbar; with a local reference the source
// site's density deviation nsrc[s] = n(s) - nbar enters as w_i nsrc[s].
template <int LAT, class ST, class CT, bool V>
__device__ __forceinline__ P2<CT> pull_site(const ST *__restrict__ src, int gx, int gy, int gz, int nx, int ny,
                                            int nz, int64_t N, P2<CT> scale, P2<CT> inv_scale, P2<CT> *v,
                                            const float2 *__restrict__ nsrc = nullptr) {
  using L = Lattice<LAT>;
  // source coordinate for velocity component c is g - c
  const int X[3] = {wrapi(gx + 1, nx), gx, wrapi(gx - 1, nx)};
  const int Y[3] = {wrapi(gy + 1, ny), gy, wrapi(gy - 1, ny)};
  const int Z[3] = {wrapi(gz + 1, nz), gz, wrapi(gz - 1, nz)};
  P2<CT> sum = pbc(CT(0));
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const int site = X[cx + 1] + nx * (Y[cy + 1] + ny * Z[cz + 1]);
    P2<CT> g = Codec2<ST, CT>::template load<false>(src + ((int64_t)i * N + site) * 2, inv_scale);
    if constexpr (local_ref<ST>()) {
      const float2 ns = __ldg(nsrc + site);
      g = pfma(wpair<LAT, ST, CT>(i, scale), pset(CT(ns.x), CT(ns.y)), g);
    }
    if (V) v[i] = g;
    sum = padd(sum, g);
  }
  return unscale<ST, CT>(sum, inv_scale);
}

// L1 prefetch of the Q population pairs a pull of site (gx, gy, gz) reads (a hint: no register
// holds the data, and the addresses are the pull's own, wrapped periodically).
template <int LAT, class ST>
__device__ __forceinline__ void prefetch_site(const ST *src, int gx, int gy, int gz, int nx, int ny, int nz,
                                              int64_t N) {
  using L = Lattice<LAT>;
  const int X[3] = {wrapi(gx + 1, nx), gx, wrapi(gx - 1, nx)};
  const int Y[3] = {wrapi(gy + 1, ny), gy, wrapi(gy - 1, ny)};
  const int Z[3] = {wrapi(gz + 1, nz), gz, wrapi(gz - 1, nz)};
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int site = X[L::c(i, 0) + 1] + nx * (Y[L::c(i, 1) + 1] + ny * Z[L::c(i, 2) + 1]);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(src + ((int64_t)i * N + site) * 2));
  }
}

// psi(n) - psi(nbar) per component; for psi = exp(-1/n): psibar * expm1((n - nbar) / (n nbar)).
// psi of a component enters only its own self-coupling force term (Eq. sc_force), so a component
// with G_JJ = 0 (gself 0) gets 0 instead: its force term is 0 either way, and the division and
// expm1 are skipped (the branch is uniform: the couplings are the lattice's).
template <class CT>
__device__ __forceinline__ P2<CT> psi_deviation(P2<CT> dn, P2<CT> nbar, P2<CT> psibar, int psi_exp, P2<CT> gself) {
  if (!psi_exp) return dn;
  const P2<CT> n = padd(nbar, dn);
  const P2<CT> q = pmul(n, nbar);
  const CT ex = gself.x != CT(0) ? expm1_ct(rdiv(dn.x, q.x)) : CT(0);
  const CT ey = gself.y != CT(0) ? expm1_ct(rdiv(dn.y, q.y)) : CT(0);
  return pmul(psibar, pset(ex, ey));
}

// Shared-memory bytes of one block: density and psi deviation pairs, a ring of
// planes of (32 + 2 HALO) x (TY + 2 HALO) sites.
template <int LAT, int STEN, class CT, int TY>
constexpr size_t step_smem_bytes() {
  constexpr int H = Stencil<LAT, STEN>::HALO;
  constexpr int HZ = (LAT == kD3Q19) ? H : 0;
  constexpr int NPL = (HZ == 0) ? 1 : 2 * HZ + 2;
  return sizeof(P2<CT>) * 2 * NPL * (32 + 2 * H) * (TY + 2 * H);
}

// ---- the collision (Eqs. sc_force, u, feq, Guo, omega_i, lbm) on component pairs
// Ring layout: s_dn / s_psi [NPL][PLANE] pairs, PLANE = (32 + 2 HALO) x (TY + 2 HALO);
// sl[d] is the ring slot of plane c - HZ + d.

// Forces (Eq. sc_force):
//   F_A = -G c_s^2 n_A sum_a W xi_a n_B(x + xi_a) - G_AA c_s^2 psi_A sum_a W xi_a psi_A(x + xi_a)
//   F_B = (A <-> B),
// each +/- stencil pair taken as one difference of deviations.
template <int LAT, int STEN, class CT, int TY>
__device__ __forceinline__ void force_pair(const StepArgs<CT> &a, const P2<CT> *s_dn, const P2<CT> *s_psi,
                                           const int *sl, int own, P2<CT> n, P2<CT> psi, P2<CT> (&F)[3]) {
  using SN = Stencil<LAT, STEN>;
  constexpr int H = SN::HALO;
  constexpr int HZ = (LAT == kD3Q19) ? H : 0;
  constexpr int SX = 32 + 2 * H;
  constexpr int PLANE = SX * (TY + 2 * H);
  P2<CT> S[3] = {pbc(CT(0)), pbc(CT(0)), pbc(CT(0))}, T[3] = {pbc(CT(0)), pbc(CT(0)), pbc(CT(0))};
#pragma unroll
  for (int k = 0; k < SN::NH; ++k) {
    const int vx = SN::v(k, 0), vy = SN::v(k, 1), vz = SN::v(k, 2);
    const int ip = own + vy * SX + vx, im = own - vy * SX - vx;
    const int zp = sl[HZ + vz] * PLANE, zm = sl[HZ - vz] * PLANE;
    const P2<CT> d = psub(s_dn[zp + ip], s_dn[zm + im]);
    if (vx) S[0] = pfma(pbc(CT(SN::W(k) * vx)), d, S[0]);
    if (vy) S[1] = pfma(pbc(CT(SN::W(k) * vy)), d, S[1]);
    if (vz) S[2] = pfma(pbc(CT(SN::W(k) * vz)), d, S[2]);
    if (a.self_on) {
      const P2<CT> e = psub(s_psi[zp + ip], s_psi[zm + im]);
      if (vx) T[0] = pfma(pbc(CT(SN::W(k) * vx)), e, T[0]);
      if (vy) T[1] = pfma(pbc(CT(SN::W(k) * vy)), e, T[1]);
      if (vz) T[2] = pfma(pbc(CT(SN::W(k) * vz)), e, T[2]);
    }
  }
  // cross term: component A feels the gradient of n_B and vice versa
  const P2<CT> cn = pmul(pbc(a.gcross), n), cp = pmul(a.gself, psi);
#pragma unroll
  for (int m = 0; m < 3; ++m) F[m] = pfma(cp, T[m], pmul(cn, pswap(S[m])));
}

// Momentum sums j_J = sum_i g_i xi_i (step units) from opposite-pair differences.
template <int LAT, class CT>
__device__ __forceinline__ void momentum_sums(const P2<CT> *g, P2<CT> (&j)[3]) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  P2<CT> d[Q];
#pragma unroll
  for (int i = 1; i < Q; i += 2) d[i] = psub(g[i], g[i + 1]);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    P2<CT> acc = pbc(CT(0));
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int cm = L::c(i, m);
      if (cm > 0) acc = padd(acc, d[i]);
      if (cm < 0) acc = psub(acc, d[i]);
    }
    j[m] = acc;
  }
}

// Half momenta h_J = j_J + F_J / 2.
template <class ST, class CT>
__device__ __forceinline__ void half_momentum(const P2<CT> (&j)[3], const P2<CT> (&F)[3], P2<CT> inv_scale,
                                              P2<CT> (&h)[3]) {
#pragma unroll
  for (int m = 0; m < 3; ++m) h[m] = pfma(pbc(CT(0.5)), F[m], unscale<ST, CT>(j[m], inv_scale));
}

// What a site's collision needs of its own arriving populations.  In general the
// population pairs themselves (CARRY = Q pairs).  With tau_A = tau_B = 1 (T1) the
// relaxation keeps nothing of them, (1 - 1/tau) f_i = 0, and only their momentum
// sums enter (CARRY = 3 pairs): the kernels then keep those across the planes between
// a site's sum and its collision, and the stored results are the same bits.
template <int LAT, bool T1>
__host__ __device__ constexpr int carry_size() {
  return T1 ? 3 : Lattice<LAT>::Q;
}
// The carry of a site from its arriving pairs g (step units).
template <int LAT, class CT, bool T1>
__device__ __forceinline__ void make_carry(const P2<CT> (&g)[Lattice<LAT>::Q], P2<CT> (&c)[carry_size<LAT, T1>()]) {
  if constexpr (T1) {
    momentum_sums<LAT, CT>(g, c);
  } else {
#pragma unroll
    for (int i = 0; i < Lattice<LAT>::Q; ++i) c[i] = g[i];
  }
}

// Common velocity of Eq. u: n u = h_A + h_B.
template <class CT>
__device__ __forceinline__ void common_velocity(const P2<CT> (&h)[3], P2<CT> n, CT (&u)[3]) {
  const CT inv_n = rdiv(CT(1), radd(n.x, n.y));
#pragma unroll
  for (int m = 0; m < 3; ++m) u[m] = rmul(radd(h[m].x, h[m].y), inv_n);
}

// BGK + Guo in pair form.  With omega = 1/tau, gamma = 1 - 1/(2 tau):
//   f* = (1 - omega) f + omega f^eq + gamma F_i
//      = (1 - omega) f + w_i [a0 + a2 cu^2 + a3 cu cF  +/-  (a1 cu + a4 cF)]
// with cu = xi.u, cF = xi.F for the "+" member of an opposite pair and
//   a0 = omega dn - 1.5 omega n u.u - 3 gamma u.F, a1 = 3 omega n,
//   a2 = 4.5 omega n, a3 = 9 gamma, a4 = 3 gamma
// (Eq. feq with c_s^2 = 1/3 written as a deviation from w_i nbar, and Eq. Guo).
// T1 (tau_A = tau_B = 1): keep = 1 - omega = 0 and g is not read (fma(0, g, x) = x).
template <int LAT, class ST, class CT, bool T1>
__device__ __forceinline__ void collide_pair(const StepArgs<CT> &a, const P2<CT> *g, P2<CT> n, P2<CT> dn,
                                             const CT (&u)[3], const P2<CT> (&F)[3],
                                             P2<CT> (&out)[Lattice<LAT>::Q]) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  const P2<CT> om = a.omega, ga = a.guo;
  const CT uu = rfma(u[2], u[2], rfma(u[1], u[1], rmul(u[0], u[0])));
  const P2<CT> uF = pfma(pbc(u[2]), F[2], pfma(pbc(u[1]), F[1], pmul(pbc(u[0]), F[0])));
  // with a local reference the stored value is out_i - w_i dn (see store_pairs): the - dn is taken
  // into a0 here, (omega - 1) dn in place of omega dn (zero for tau = 1)
  const P2<CT> a0 = pfma(pmul(pbc(CT(-3)), ga), uF,
                         pfma(pmul(pmul(pbc(CT(-1.5)), om), n), pbc(uu),
                              pmul(local_ref<ST>() ? psub(om, pbc(CT(1))) : om, dn)));
  const P2<CT> a1 = pmul(pmul(pbc(CT(3)), om), n), a2 = pmul(pmul(pbc(CT(4.5)), om), n);
  const P2<CT> a3 = pmul(pbc(CT(9)), ga), a4 = pmul(pbc(CT(3)), ga);
  const P2<CT> keep = psub(pbc(CT(1)), om);
  out[0] = T1 ? pmul(wpair<LAT, ST, CT>(0, a.scale), a0) : pfma(keep, g[0], pmul(wpair<LAT, ST, CT>(0, a.scale), a0));
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int c[3] = {L::c(i, 0), L::c(i, 1), L::c(i, 2)};
    const P2<CT> w = wpair<LAT, ST, CT>(i, a.scale);
    CT cu = CT(0);
    P2<CT> cF = pbc(CT(0));
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      if (c[m] > 0) { cu = radd(cu, u[m]); cF = padd(cF, F[m]); }
      if (c[m] < 0) { cu = rsub(cu, u[m]); cF = psub(cF, F[m]); }
    }
    const P2<CT> cu2 = pbc(cu);
    const P2<CT> E = pfma(cu2, pfma(pmul(w, a2), cu2, pmul(pmul(w, a3), cF)), pmul(w, a0));
    const P2<CT> O = pfma(pmul(w, a1), cu2, pmul(pmul(w, a4), cF));
    if constexpr (T1) {
      out[i] = padd(E, O);
      out[i + 1] = psub(E, O);
    } else {
      out[i] = pfma(keep, g[i], padd(E, O));
      out[i + 1] = pfma(keep, g[i + 1], psub(E, O));
    }
  }
}

// Status: a non-finite density, or a non-positive one while psi = exp(-1/n) is in use.
template <class CT>
__device__ __forceinline__ void check_density(const StepArgs<CT> &a, P2<CT> n) {
  const bool finite = fabs(n.x + n.y) < CT(INFINITY);
  const bool positive = n.x > CT(0) && n.y > CT(0);
  if (!finite || (a.self_on && a.psi_exp && !positive)) atomicOr(a.err, 1u);
}

// Store the post-collision pairs (deviations from w_i nbar).  With a local
// reference the stored value is relative to this site's density n = nbar + dn,
// i.e. out_i - w_i dn (collide_pair has already subtracted w_i dn), and
// dn = n - nbar goes to ndst.
template <int LAT, class ST, class CT, int Q>
__device__ __forceinline__ void store_pairs(const StepArgs<CT> &a, ST *__restrict__ dst, int64_t site,
                                            const P2<CT> (&out)[Q], P2<CT> n, P2<CT> dn) {
#pragma unroll
  for (int i = 0; i < Q; ++i) Codec2<ST, CT>::store(dst + ((int64_t)i * a.N + site) * 2, out[i], a.scale);
  if constexpr (local_ref<ST>()) a.ndst[site] = make_float2(float(dn.x), float(dn.y));
}

// Collision of one site from the carry of its arriving population pairs and the ring.
template <int LAT, int STEN, class ST, class CT, int TY, bool T1>
__device__ __forceinline__ void collide_site(const StepArgs<CT> &a, const P2<CT> (&carry)[carry_size<LAT, T1>()],
                                             const P2<CT> *s_dn, const P2<CT> *s_psi, const int *sl, int own,
                                             bool valid, ST *__restrict__ dst, int64_t site) {
  constexpr int Q = Lattice<LAT>::Q;
  constexpr int HZ = (LAT == kD3Q19) ? Stencil<LAT, STEN>::HALO : 0;
  constexpr int H = Stencil<LAT, STEN>::HALO;
  constexpr int PLANE = (32 + 2 * H) * (TY + 2 * H);
  const P2<CT> dn = s_dn[sl[HZ] * PLANE + own];
  const P2<CT> n = padd(a.nbar, dn);
  const P2<CT> psi = a.self_on ? padd(a.psibar, s_psi[sl[HZ] * PLANE + own]) : pbc(CT(0));
  P2<CT> F[3], j[3], h[3], out[Q];
  CT u[3];
  force_pair<LAT, STEN, CT, TY>(a, s_dn, s_psi, sl, own, n, psi, F);
  if constexpr (T1) {
#pragma unroll
    for (int m = 0; m < 3; ++m) j[m] = carry[m];
  } else {
    momentum_sums<LAT, CT>(carry, j);
  }
  half_momentum<ST, CT>(j, F, a.inv_scale, h);
  common_velocity<CT>(h, n, u);
  collide_pair<LAT, ST, CT, T1>(a, carry, n, dn, u, F, out);
  if (valid) {
    check_density<CT>(a, n);
    store_pairs<LAT, ST, CT, Q>(a, dst, site, out, n, dn);
  }
}

// The work of this block of a single-lattice launch: column (bx, by) of 32 x TY
// sites, planes z0 .. zend - 1.  Balanced z split (a.zbal_k > 0; a 1-D grid of
// K C + R blocks over the C = zbal_cols columns): chunk j of column c, columns c < R
// cut into K + 1 equal z-chunks, the others into K, in chunk-major order.  Else the
// 3-D grid of columns (blockIdx.x, blockIdx.y) and tile_z-plane chunks blockIdx.z.
// In the balanced split odd chunks march down (down = true): all chunks of a column
// run in the same wave or two, and the z-halo planes two neighbouring chunks share
// are then read by both at the same time (both at their start or both at their end),
// from L2 once, instead of a whole chunk duration apart (128^3 F32 +1.2 %, E6 slab
// +1.8 %).  The 3-D grid runs chunk after chunk in many waves: there a chunk that
// starts where the previous wave's chunk ended finds its halo planes in L2, so every
// chunk marches up (alternating there measured 1 % slower at 256^3).
template <class CT>
__device__ __forceinline__ void block_work(const StepArgs<CT> &a, int &bx, int &by, int &z0, int &zend,
                                           bool &down) {
  if (a.zbal_k > 0) {
    const int b = blockIdx.x, C = a.zbal_cols, K = a.zbal_k;
    int j, c;
    if (b < K * C) {
      j = b / C;
      c = b - j * C;
    } else {
      j = K;
      c = b - K * C;
    }
    const int kc = K + (c < a.zbal_rem ? 1 : 0);
    z0 = (int)((int64_t)j * a.nz / kc);
    zend = (int)((int64_t)(j + 1) * a.nz / kc);
    by = c / a.zbal_cols_x;
    bx = c - by * a.zbal_cols_x;
    down = (j & 1) != 0;
  } else {
    bx = blockIdx.x;
    by = blockIdx.y;
    z0 = blockIdx.z * a.tile_z;
    zend = min(z0 + a.tile_z, a.nz);
    down = false;
  }
}

// One block's work: the column (bx, by), planes z0 .. zend - 1, of the lattice described by a,
// marched upward or (down) downward.
template <int LAT, int STEN, class ST, class CT, int TY, bool T1>
__device__ __forceinline__ void step_block(const StepArgs<CT> &a, int bx, int by, int z0, int zend, bool down,
                                           unsigned char *smem_raw) {
  using L = Lattice<LAT>;
  using SN = Stencil<LAT, STEN>;
  constexpr int Q = L::Q;
  constexpr int H = SN::HALO;
  constexpr int HZ = (LAT == kD3Q19) ? H : 0;
  constexpr int NPL = (HZ == 0) ? 1 : 2 * HZ + 2;  // ring planes: one barrier per plane
  constexpr int SX = 32 + 2 * H, SY = TY + 2 * H;
  constexpr int PLANE = SX * SY;
  constexpr int NHALO = PLANE - 32 * TY;
  constexpr int NT = 32 * TY;
  // a site's carry (its own populations, or with T1 their momentum sums) stays in registers
  // from its sum to its collision HZ planes later; the general E6 form pulls the site again
  constexpr bool KEEP = T1 || (HZ <= 1);
  constexpr int CQ = carry_size<LAT, T1>();
  constexpr int NC = KEEP ? HZ + 1 : 1;  // carries in flight: planes m - HZ .. m

  P2<CT> *s_dn = reinterpret_cast<P2<CT> *>(smem_raw);  // [NPL][PLANE]
  P2<CT> *s_psi = s_dn + NPL * PLANE;                   // [NPL][PLANE]

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t N = a.N;
  const int x0 = bx * 32, y0 = by * TY;
  const ST *__restrict__ src = static_cast<const ST *>(a.src);
  ST *__restrict__ dst = static_cast<ST *>(a.dst);

  const bool valid_xy = (x0 + tx < nx) && (y0 + ty < ny);
  const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
  const int own = (ty + H) * SX + (tx + H);

  P2<CT> car[NC][CQ];
  int slot = 0;
  const int np = zend - z0 + 2 * HZ;  // planes z0 - HZ .. zend - 1 + HZ, in march order m
  for (int m = 0; m < np; ++m) {
    const int p = down ? zend - 1 + HZ - m : z0 - HZ + m;
    const int gz = ((p % nz) + nz) % nz;
    if constexpr (NHALO <= NT) {
      // ---- density / psi deviations of this plane: own site and (threads tid < NHALO) one halo
      // site, both pulls issued before either sum is used so that their L2 latencies overlap;
      // threads without a halo site pull their own site a second time and discard it
      const bool hal = tid < NHALO;
      int px = 0, py = 0;
      if (tid < 2 * H * SX) {
        const int r = tid / SX;
        px = tid - r * SX - H;
        py = r < H ? r - H : TY + (r - H);
      } else {
        const int k = tid - 2 * H * SX, r = k / (2 * H), c = k - r * (2 * H);
        py = r;
        px = c < H ? c - H : 32 + (c - H);
      }
      const int hx = hal ? ((x0 + px) % nx + nx) % nx : gx, hy = hal ? ((y0 + py) % ny + ny) % ny : gy;
      const int idx = (py + H) * SX + (px + H);
      P2<CT> g[Q];
      const P2<CT> dn =
          pull_site<LAT, ST, CT, KEEP>(src, gx, gy, gz, nx, ny, nz, N, a.scale, a.inv_scale, g, a.nsrc);
      const P2<CT> dh =
          pull_site<LAT, ST, CT, false>(src, hx, hy, gz, nx, ny, nz, N, a.scale, a.inv_scale, nullptr, a.nsrc);
      s_dn[slot * PLANE + own] = dn;
      if (hal) s_dn[slot * PLANE + idx] = dh;
      if (a.self_on) {
        const P2<CT> pn = psi_deviation<CT>(dn, a.nbar, a.psibar, a.psi_exp, a.gself);
        const P2<CT> ph = psi_deviation<CT>(dh, a.nbar, a.psibar, a.psi_exp, a.gself);
        s_psi[slot * PLANE + own] = pn;
        if (hal) s_psi[slot * PLANE + idx] = ph;
      }
      if constexpr (KEEP) {
#pragma unroll
        for (int q = 0; q + 1 < NC; ++q)
#pragma unroll
          for (int i = 0; i < CQ; ++i) car[q][i] = car[q + 1][i];
        make_carry<LAT, CT, T1>(g, car[NC - 1]);
      }
    } else {
      // ---- density / psi deviations of this plane: own site
      {
        P2<CT> g[Q];
        const P2<CT> dn =
            pull_site<LAT, ST, CT, KEEP>(src, gx, gy, gz, nx, ny, nz, N, a.scale, a.inv_scale, g, a.nsrc);
        s_dn[slot * PLANE + own] = dn;
        if (a.self_on) s_psi[slot * PLANE + own] = psi_deviation<CT>(dn, a.nbar, a.psibar, a.psi_exp, a.gself);
        if constexpr (KEEP) {
#pragma unroll
          for (int q = 0; q + 1 < NC; ++q)
#pragma unroll
            for (int i = 0; i < CQ; ++i) car[q][i] = car[q + 1][i];
          make_carry<LAT, CT, T1>(g, car[NC - 1]);
        }
      }
      // ---- halo sites (full rows first, for coalescing, then the side columns)
      for (int h = tid; h < NHALO; h += NT) {
        int px, py;
        if (h < 2 * H * SX) {
          const int r = h / SX;
          px = h - r * SX - H;
          py = r < H ? r - H : TY + (r - H);
        } else {
          const int k = h - 2 * H * SX, r = k / (2 * H), c = k - r * (2 * H);
          py = r;
          px = c < H ? c - H : 32 + (c - H);
        }
        const int hx = ((x0 + px) % nx + nx) % nx, hy = ((y0 + py) % ny + ny) % ny;
        const P2<CT> dn =
            pull_site<LAT, ST, CT, false>(src, hx, hy, gz, nx, ny, nz, N, a.scale, a.inv_scale, nullptr, a.nsrc);
        const int idx = (py + H) * SX + (px + H);
        s_dn[slot * PLANE + idx] = dn;
        if (a.self_on) s_psi[slot * PLANE + idx] = psi_deviation<CT>(dn, a.nbar, a.psibar, a.psi_exp, a.gself);
      }
    }
    __syncthreads();
    if constexpr (HZ >= 2) {
      // E6: the own site's pulls of the next plane go to L1 while this plane collides (E6 slab
      // 81.9 -> 80.3 us; the same hint costs E4 at 128^3 1.5 %, and the halo site's pulls as well
      // cost E6 9 %)
      if (m + 1 < np) {
        const int pn = down ? zend - 2 + HZ - m : z0 - HZ + m + 1;
        prefetch_site<LAT, ST>(src, gx, gy, ((pn % nz) + nz) % nz, nx, ny, nz, N);
      }
    }

    // ---- collide plane c (march position m - HZ) once planes c - HZ .. c + HZ are in the ring
    if (m >= 2 * HZ) {
      const int c = down ? p + HZ : p - HZ;
      int sl[2 * HZ + 1];  // ring slot of plane c - HZ + d, at march position m - 2 HZ + d (m - d down)
#pragma unroll
      for (int d = 0; d <= 2 * HZ; ++d) sl[d] = (down ? slot - d + NPL : slot - 2 * HZ + d + 2 * NPL) % NPL;
      const int gzc = ((c % nz) + nz) % nz;
      const int64_t site = (int64_t)gx + (int64_t)nx * (gy + (int64_t)ny * gzc);
      if constexpr (KEEP) {
        collide_site<LAT, STEN, ST, CT, TY, T1>(a, car[0], s_dn, s_psi, sl, own, valid_xy, dst, site);
      } else {
        P2<CT> g[Q];
        pull_site<LAT, ST, CT, true>(src, gx, gy, gzc, nx, ny, nz, N, a.scale, a.inv_scale, g, a.nsrc);
        collide_site<LAT, STEN, ST, CT, TY, T1>(a, g, s_dn, s_psi, sl, own, valid_xy, dst, site);
      }
    }
    slot = (slot + 1 == NPL) ? 0 : slot + 1;
  }
}

// T1: the tau_A = tau_B = 1 form (see carry_size).
template <int LAT, int STEN, class ST, class CT, int TY, bool T1>
__global__ void __launch_bounds__(32 * TY, (TY >= 16 ? 1 : 16 / TY)) sc_step_kernel(const StepArgs<CT> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int bx, by, z0, zend;
  bool down;
  block_work(a, bx, by, z0, zend, down);
  step_block<LAT, STEN, ST, CT, TY, T1>(a, bx, by, z0, zend, down, smem_raw);
}

// Batched form: one launch steps several lattices.  Block b works on item
// items[b] = (lattice, bx, by, bz); lattice l's arguments are args[l] (read
// from global memory), with source and destination swapped when swap != 0.
template <int LAT, int STEN, class ST, class CT, int TY, bool T1>
__global__ void __launch_bounds__(32 * TY, (TY >= 16 ? 1 : 16 / TY))
    sc_step_batched(const StepArgs<CT> *__restrict__ args, const int4 *__restrict__ items, int swap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int4 it = items[blockIdx.x];
  StepArgs<CT> a = args[it.x];
  if (swap) {
    const void *t = a.src;
    a.src = a.dst;
    a.dst = const_cast<void *>(t);
    const float2 *u = a.nsrc;
    a.nsrc = a.ndst;
    a.ndst = const_cast<float2 *>(u);
  }
  const int z0 = it.w * a.tile_z;
  step_block<LAT, STEN, ST, CT, TY, T1>(a, it.y, it.z, z0, min(z0 + a.tile_z, a.nz), false, smem_raw);
}

}  // namespace scgb
