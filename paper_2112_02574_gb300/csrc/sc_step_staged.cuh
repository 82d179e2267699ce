// The fused time step, staged variant (D3Q19, E4 stencil, nx % 32 == 0,
// nx >= 64).  Same arithmetic as sc_step_kernel (shared collide_site and the
// same summation order), different data movement:
//
//  * A block owns a column of 32 x TY sites in x-y and tile_z planes in z
//    (blocks in x, y, z-chunk order, so neighbouring columns run together and
//    the rows they share are L2 hits) and marches along z.
//  * For every plane z the block needs, per direction i, the source rows
//    f*_i(., y - c_i^y, z - c_i^z) (both components, interleaved) for the tile
//    rows plus one halo row on each side, over the 16-byte aligned x window
//    [x0 - OFF, x0 + 32 + OFF).  All threads copy these windows in 16-byte
//    chunks with cp.async (each chunk wraps periodically on its own, since
//    nx * pair size is a multiple of 16) into a two-stage shared-memory
//    pipeline, one commit group per plane: the copies for plane k + 2 are in
//    flight while plane k is summed and plane k - 1 is collided.
//  * Densities of tile + halo are summed from the staged rows into the same
//    ring of deviation planes the generic kernel uses; the own site's
//    populations move to registers, which frees the stage for the next copy.
//  * Waiting is cp.async.wait_group plus block barriers; no block waits on
//    another block.
#pragma once

#include "sc_step_kernel.cuh"

namespace scgb {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <class ST, int TY>
struct StagedGeom {
  static constexpr int Q = 19;
  static constexpr int RY = TY + 2;                      // tile rows + one halo row each side
  static constexpr int CE = 16 / (2 * int(sizeof(ST)));  // sites per 16-byte chunk
  static constexpr int OFF = CE < 2 ? 2 : CE;            // window margin (halo pulls reach 2 sites), in sites
  static constexpr int WX = 32 + 2 * OFF;                // window width, sites
  static constexpr int STAGE_ELEMS = Q * RY * WX * 2;    // [i][row][x][J]
  static constexpr int STAGE_BYTES = STAGE_ELEMS * int(sizeof(ST));
  static constexpr int SX = 34, SY = TY + 2, PLANE = SX * SY, NPL = 4;
  static constexpr int NHALO = PLANE - 32 * TY;
  static constexpr int NCH = WX / CE;              // chunks per row window
  static constexpr int NROW = Q * RY;              // row windows per plane
};

// Shared memory: two stages, per-plane row source pointers, row tables, density / psi rings.
template <class ST, class CT, int TY>
constexpr size_t staged_smem_bytes() {
  using G = StagedGeom<ST, TY>;
  return 2 * size_t(G::STAGE_BYTES) + sizeof(int64_t) * 2 * G::NROW + sizeof(int) * ((G::NROW + 3) & ~3) +
         sizeof(P2<CT>) * 2 * G::NPL * G::PLANE;
}

// Sum of the Q staged population pairs arriving at tile position (px, py), in
// direction order (identical to pull_site's order); values go to v[] when V is true.
template <class ST, class CT, int TY, bool V>
__device__ __forceinline__ P2<CT> staged_sum(const ST *stage, int px, int py, const P2<CT> *inv_scale, P2<CT> *v) {
  using G = StagedGeom<ST, TY>;
  using L = Lattice<kD3Q19>;
  const ST *base = stage + ((py + 1) * G::WX + px + G::OFF) * 2;
  P2<CT> sum = pbc(CT(0));
#pragma unroll
  for (int i = 0; i < G::Q; ++i) {
    const P2<CT> g =
        Codec2<ST, CT>::template load<true>(base + (i * G::RY * G::WX - L::c(i, 0)) * 2, inv_scale[i]);
    if (V) v[i] = g;
    sum = padd(sum, g);
  }
  return sum;
}

template <class ST, class CT, int TY>
__global__ void __launch_bounds__(32 * TY, 1) sc_step_staged(const StepArgs<CT> a) {
  using G = StagedGeom<ST, TY>;
  using L = Lattice<kD3Q19>;
  constexpr int Q = G::Q;
  constexpr int NT = 32 * TY;
  constexpr int NTASK = (G::NHALO + NT - 1) / NT;  // halo sums per thread and plane
  extern __shared__ __align__(128) unsigned char smem_raw[];
  ST *stage0 = reinterpret_cast<ST *>(smem_raw);                                       // [2][STAGE_ELEMS]
  const ST **rowsrc = reinterpret_cast<const ST **>(smem_raw + 2 * G::STAGE_BYTES);    // [NROW] this plane's rows
  int64_t *rowbase = reinterpret_cast<int64_t *>(rowsrc + G::NROW);                    // [NROW]
  int *rowcz = reinterpret_cast<int *>(rowbase + G::NROW);                             // [NROW]
  P2<CT> *s_dn = reinterpret_cast<P2<CT> *>(rowcz + ((G::NROW + 3) & ~3));           // [NPL][PLANE]
  P2<CT> *s_psi = s_dn + G::NPL * G::PLANE;                                            // [NPL][PLANE]

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t plane_elems = (int64_t)nx * ny;
  const ST *__restrict__ src = static_cast<const ST *>(a.src);
  ST *__restrict__ dst = static_cast<ST *>(a.dst);
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY, z0 = blockIdx.z * a.tile_z;
  const int zend = min(z0 + a.tile_z, nz);
  const int np = zend - z0 + 2;  // planes z0 - 1 .. zend
  const int own = (ty + 1) * G::SX + (tx + 1);
  const bool valid_xy = (y0 + ty < ny);  // x tiles are full (nx % 32 == 0)
  const int gx = x0 + tx, gy = (y0 + ty) % ny;

  // row tables of this column: row = i * RY + r holds the source row
  // y0 - 1 + r - c_i^y of direction i (both components); the plane part follows per copy
  for (int row = tid; row < G::NROW; row += NT) {
    const int i = row / G::RY, r = row - i * G::RY;
    int cy = 0, cz = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q == i) {
        cy = L::c(q, 1);
        cz = L::c(q, 2);
      }
    int ys = y0 - 1 + r - cy;
    ys = ((ys % ny) + ny) % ny;
    rowbase[row] = ((int64_t)i * a.N + (int64_t)ys * nx) * 2;
    rowcz[row] = cz;
  }
  // this thread's halo sums (fixed for the whole column)
  int task_idx[NTASK], task_px[NTASK], task_py[NTASK];
  bool task_on[NTASK];
#pragma unroll
  for (int m = 0; m < NTASK; ++m) {
    const int h = tid + m * NT;
    task_on[m] = h < G::NHALO;
    int px = 0, py = 0;
    if (h < 2 * G::SX) {
      const int r = h / G::SX;
      px = h - r * G::SX - 1;
      py = r == 0 ? -1 : TY;
    } else if (h < G::NHALO) {
      const int k2 = h - 2 * G::SX;
      py = k2 >> 1;
      px = (k2 & 1) ? 32 : -1;
    }
    task_px[m] = px;
    task_py[m] = py;
    task_idx[m] = (py + 1) * G::SX + (px + 1);
  }
  auto wrapz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
  // source row pointers of plane z (direction with c^z = +1 reads plane z - 1, and so on)
  auto rows_for = [&](int z) {
    const int64_t zo_p = (int64_t)wrapz(z + 1) * plane_elems * 2, zo_0 = (int64_t)z * plane_elems * 2,
                  zo_m = (int64_t)wrapz(z - 1) * plane_elems * 2;
    for (int row = tid; row < G::NROW; row += NT) {
      const int cz = rowcz[row];
      rowsrc[row] = src + rowbase[row] + (cz > 0 ? zo_m : (cz < 0 ? zo_p : zo_0));
    }
  };
  // copies of the rows in rowsrc into stage s: 16-byte chunks, linear over (row, chunk)
  auto copy_rows = [&](int s) {
    ST *stage = stage0 + s * G::STAGE_ELEMS;
    for (int t = tid; t < G::NROW * G::NCH; t += NT) {
      const int row = t / G::NCH, c = t - row * G::NCH;
      int xs = x0 - G::OFF + c * G::CE;
      xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
      cp_async16(stage + (row * G::WX + c * G::CE) * 2, rowsrc[row] + (int64_t)xs * 2);
    }
  };
  __syncthreads();
  rows_for(wrapz(z0 - 1));
  __syncthreads();
  copy_rows(0);
  cp_async_commit();
  __syncthreads();
  rows_for(wrapz(z0));
  __syncthreads();
  copy_rows(1);
  cp_async_commit();

  // one plane of the march: sum plane k (own population pairs into `mine`),
  // then collide plane k - 1 from `prev`
  auto body = [&](int k, P2<CT> (&prev)[Q], P2<CT> (&mine)[Q]) {
    const int s = k & 1;
    const ST *stage = stage0 + s * G::STAGE_ELEMS;
    cp_async_wait_one();  // all groups but the newest (plane k + 1) are complete: plane k is in
    __syncthreads();      // ... and visible to every thread; the last copy pass is over
    if (k + 2 < np) rows_for(wrapz(z0 + 1 + k));
    const int slot = k & (G::NPL - 1);
    {
      const P2<CT> dn = staged_sum<ST, CT, TY, true>(stage, tx, ty, a.inv_scale, mine);
      s_dn[slot * G::PLANE + own] = dn;
      if (a.self_on) s_psi[slot * G::PLANE + own] = psi_deviation<CT>(dn, a.nbar, a.psibar, a.psi_exp);
    }
#pragma unroll
    for (int m = 0; m < NTASK; ++m) {
      if (task_on[m]) {
        const P2<CT> dn = staged_sum<ST, CT, TY, false>(stage, task_px[m], task_py[m], a.inv_scale, nullptr);
        s_dn[slot * G::PLANE + task_idx[m]] = dn;
        if (a.self_on) s_psi[slot * G::PLANE + task_idx[m]] = psi_deviation<CT>(dn, a.nbar, a.psibar, a.psi_exp);
      }
    }
    __syncthreads();  // stage s fully read, ring plane and next row pointers written
    if (k + 2 < np) copy_rows(s);
    cp_async_commit();  // (possibly empty) group for plane k + 2 keeps "newest = next plane"
    if (k >= 2) {
      const int sl[3] = {(slot + 2) & 3, (slot + 3) & 3, slot};  // planes k-2, k-1, k
      const int c = z0 - 2 + k;
      const int64_t site = (int64_t)gx + (int64_t)nx * (gy + (int64_t)ny * c);
      collide_site<kD3Q19, kE4, ST, CT, TY>(a, prev, s_dn, s_psi, sl, own, valid_xy, dst, site);
    }
  };
  P2<CT> A[Q], B[Q];
  int k = 0;
  for (; k + 1 < np; k += 2) {
    body(k, B, A);
    body(k + 1, A, B);
  }
  if (k < np) body(k, B, A);
}

}  // namespace scgb
