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
// pulls again; populations are stored as deviations g = f - w_i nbar_J.
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

// Pull the Q populations of component J arriving at site (gx, gy, gz) and
// return their sum (the density deviation); values go to v[] when V is true.
template <int LAT, class ST, class CT, bool V>
__device__ __forceinline__ CT pull_site(const ST *__restrict__ src, int J, int gx, int gy, int gz, int nx, int ny,
                                        int nz, int64_t N, const CT *inv_scale, CT *v) {
  using L = Lattice<LAT>;
  // source coordinate for velocity component c is g - c
  const int X[3] = {wrapi(gx + 1, nx), gx, wrapi(gx - 1, nx)};
  const int Y[3] = {wrapi(gy + 1, ny), gy, wrapi(gy - 1, ny)};
  const int Z[3] = {wrapi(gz + 1, nz), gz, wrapi(gz - 1, nz)};
  const ST *base = src + (int64_t)J * L::Q * N;
  CT sum = CT(0);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const int site = X[cx + 1] + nx * (Y[cy + 1] + ny * Z[cz + 1]);
    const CT g = Codec<ST, CT>::load(base + (int64_t)i * N + site, inv_scale[i]);
    if (V) v[i] = g;
    sum += g;
  }
  return sum;
}

template <class CT>
__device__ __forceinline__ CT psi_deviation(CT dn, CT nbar, CT psibar, int psi_exp) {
  // psi(n) - psi(nbar); for psi = exp(-1/n): psibar * expm1((n - nbar) / (n nbar))
  if (!psi_exp) return dn;
  const CT n = nbar + dn;
  return psibar * expm1_ct(dn / (n * nbar));
}

// Shared-memory bytes of one block: density and psi deviations, both
// components, a ring of planes of (32 + 2 HALO) x (TY + 2 HALO) sites.
template <int LAT, int STEN, class CT, int TY>
constexpr size_t step_smem_bytes() {
  constexpr int H = Stencil<LAT, STEN>::HALO;
  constexpr int HZ = (LAT == kD3Q19) ? H : 0;
  constexpr int NPL = (HZ == 0) ? 1 : 2 * HZ + 2;
  return sizeof(CT) * 2 * 2 * NPL * (32 + 2 * H) * (TY + 2 * H);
}

// Collision of one site from its arriving populations g[J][i] and the ring of
// density / psi deviation planes (Eqs. sc_force, u, feq, Guo, omega_i, lbm).
template <int LAT, int STEN, class ST, class CT, int TY>
__device__ __forceinline__ void collide_site(const StepArgs<CT> &a, const CT (&g)[2][Lattice<LAT>::Q],
                                             const CT *s_dn, const CT *s_psi, const int *sl, int own,
                                             bool valid, ST *__restrict__ dst, int64_t site) {
  using L = Lattice<LAT>;
  using SN = Stencil<LAT, STEN>;
  constexpr int Q = L::Q;
  constexpr int H = SN::HALO;
  constexpr int HZ = (LAT == kD3Q19) ? H : 0;
  constexpr int NPL = (HZ == 0) ? 1 : 2 * HZ + 2;
  constexpr int SX = 32 + 2 * H;
  constexpr int PLANE = SX * (TY + 2 * H);
  const int64_t N = a.N;
  auto DN = [&](int J, int z, int i) { return s_dn[(J * NPL + z) * PLANE + i]; };
  auto PS = [&](int J, int z, int i) { return s_psi[(J * NPL + z) * PLANE + i]; };

  CT dn[2], n[2], psi[2];
#pragma unroll
  for (int J = 0; J < 2; ++J) {
    dn[J] = DN(J, sl[HZ], own);
    n[J] = a.nbar[J] + dn[J];
    psi[J] = a.self_on ? a.psibar[J] + PS(J, sl[HZ], own) : CT(0);
  }
  // Eq. sc_force: S_J = sum_a W xi_a n_J(x + xi_a), T_J = sum_a W xi_a psi_J(x + xi_a),
  // each +/- pair taken as one difference
  CT S[2][3] = {{0, 0, 0}, {0, 0, 0}}, T[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int k = 0; k < SN::NH; ++k) {
    const int vx = SN::v(k, 0), vy = SN::v(k, 1), vz = SN::v(k, 2);
    const CT W = CT(SN::W(k));
    const int ip = own + vy * SX + vx, im = own - vy * SX - vx;
    const int zp = sl[HZ + vz], zm = sl[HZ - vz];
#pragma unroll
    for (int J = 0; J < 2; ++J) {
      const CT d = DN(J, zp, ip) - DN(J, zm, im);
      if (vx) S[J][0] += (W * CT(vx)) * d;
      if (vy) S[J][1] += (W * CT(vy)) * d;
      if (vz) S[J][2] += (W * CT(vz)) * d;
      if (a.self_on) {
        const CT e = PS(J, zp, ip) - PS(J, zm, im);
        if (vx) T[J][0] += (W * CT(vx)) * e;
        if (vy) T[J][1] += (W * CT(vy)) * e;
        if (vz) T[J][2] += (W * CT(vz)) * e;
      }
    }
  }
  CT F[2][3], j[2][3];
#pragma unroll
  for (int J = 0; J < 2; ++J) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      F[J][m] = a.gcross * n[J] * S[1 - J][m] + a.gself[J] * psi[J] * T[J][m];
      CT acc = CT(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int cm = L::c(i, m);
        if (cm > 0) acc += g[J][i];
        if (cm < 0) acc -= g[J][i];
      }
      j[J][m] = acc;
    }
  }
  CT u[3];
  const CT inv_n = CT(1) / (n[0] + n[1]);
#pragma unroll
  for (int m = 0; m < 3; ++m) u[m] = ((j[0][m] + CT(0.5) * F[0][m]) + (j[1][m] + CT(0.5) * F[1][m])) * inv_n;
  const CT uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  if (valid && !(n[0] > CT(0) && n[1] > CT(0))) atomicOr(a.err, 1u);
#pragma unroll
  for (int J = 0; J < 2; ++J) {
    const CT uF = u[0] * F[J][0] + u[1] * F[J][1] + u[2] * F[J][2];
    ST *out = dst + (int64_t)J * Q * N + site;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
      const CT w = CT(L::w(i));
      const CT cu = CT(cx) * u[0] + CT(cy) * u[1] + CT(cz) * u[2];
      const CT cF = CT(cx) * F[J][0] + CT(cy) * F[J][1] + CT(cz) * F[J][2];
      // deviation of Eq. feq from w_i nbar_J, and the Guo term
      const CT geq = w * (dn[J] + n[J] * (CT(3) * cu + CT(4.5) * cu * cu - CT(1.5) * uu));
      const CT Fi = w * (CT(3) * cF + CT(9) * cu * cF - CT(3) * uF);
      const CT gout = g[J][i] - a.omega[J] * (g[J][i] - geq) + a.guo[J] * Fi;
      if (valid) Codec<ST, CT>::store(out + (int64_t)i * N, gout, a.scale[J][i]);
    }
  }
}

template <int LAT, int STEN, class ST, class CT, int TY>
__global__ void __launch_bounds__(32 * TY, (TY >= 16 ? 1 : 16 / TY)) sc_step_kernel(const StepArgs<CT> a) {
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
  constexpr bool KEEP = (HZ <= 1);  // own populations stay in registers until collided

  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT *s_dn = reinterpret_cast<CT *>(smem_raw);  // [2][NPL][PLANE]
  CT *s_psi = s_dn + 2 * NPL * PLANE;           // [2][NPL][PLANE]

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t N = a.N;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY, z0 = blockIdx.z * a.tile_z;
  const int zend = min(z0 + a.tile_z, nz);
  const ST *__restrict__ src = static_cast<const ST *>(a.src);
  ST *__restrict__ dst = static_cast<ST *>(a.dst);

  const bool valid_xy = (x0 + tx < nx) && (y0 + ty < ny);
  const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
  const int own = (ty + H) * SX + (tx + H);

  CT cur[2][Q], nxt[2][Q];
  int slot = 0;
  for (int p = z0 - HZ; p <= zend - 1 + HZ; ++p) {
    const int gz = ((p % nz) + nz) % nz;
    // ---- density / psi deviations of this plane: own site
#pragma unroll
    for (int J = 0; J < 2; ++J) {
      const CT dn = pull_site<LAT, ST, CT, KEEP>(src, J, gx, gy, gz, nx, ny, nz, N, a.inv_scale[J], nxt[J]);
      s_dn[(J * NPL + slot) * PLANE + own] = dn;
      if (a.self_on) s_psi[(J * NPL + slot) * PLANE + own] = psi_deviation(dn, a.nbar[J], a.psibar[J], a.psi_exp);
    }
    // ---- halo sites (full rows first, for coalescing, then the side columns)
    for (int t = tid; t < 2 * NHALO; t += NT) {
      const int J = t / NHALO, h = t - J * NHALO;
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
      const CT dn = pull_site<LAT, ST, CT, false>(src, J, hx, hy, gz, nx, ny, nz, N, a.inv_scale[J], nullptr);
      const int idx = (py + H) * SX + (px + H);
      s_dn[(J * NPL + slot) * PLANE + idx] = dn;
      if (a.self_on) s_psi[(J * NPL + slot) * PLANE + idx] = psi_deviation(dn, a.nbar[J], a.psibar[J], a.psi_exp);
    }
    __syncthreads();

    // ---- collide plane c once planes c - HZ .. c + HZ are in the ring
    const int c = p - HZ;
    if (c >= z0) {
      int sl[2 * HZ + 1];
#pragma unroll
      for (int d = 0; d <= 2 * HZ; ++d) sl[d] = (slot - 2 * HZ + d + 2 * NPL) % NPL;  // plane c - HZ + d
      const int gzc = ((c % nz) + nz) % nz;
      const int64_t site = (int64_t)gx + (int64_t)nx * (gy + (int64_t)ny * gzc);
      if (HZ == 1) {
        collide_site<LAT, STEN, ST, CT, TY>(a, cur, s_dn, s_psi, sl, own, valid_xy, dst, site);
      } else {
        if (!KEEP) {
#pragma unroll
          for (int J = 0; J < 2; ++J)
            pull_site<LAT, ST, CT, true>(src, J, gx, gy, gzc, nx, ny, nz, N, a.inv_scale[J], nxt[J]);
        }
        collide_site<LAT, STEN, ST, CT, TY>(a, nxt, s_dn, s_psi, sl, own, valid_xy, dst, site);
      }
    }
    if (HZ == 1) {
#pragma unroll
      for (int J = 0; J < 2; ++J)
#pragma unroll
        for (int i = 0; i < Q; ++i) cur[J][i] = nxt[J][i];
    }
    slot = (slot + 1 == NPL) ? 0 : slot + 1;
  }
}

}  // namespace scgb
