// The fused time step, staged variant (D3Q19, E4 stencil, nx >= 32 and nx a
// multiple of the sites in a 16-byte chunk).  Same arithmetic as sc_step_kernel
// (shared collide_site and the same summation order), different data movement:
//
//  * A block owns a column of 32 x TY sites in x-y (the last x tile may be
//    partial) and tile_z planes in z
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
// 16-byte copy global -> shared, cached in L2 only; the L2::256B prefetch-size hint lets an L2
// miss fetch the whole aligned 256-byte block (a row window spans 288 B and more): same-box
// +1.0 % at 256^3 and +0.4 % at 128^3 in FP32 against no hint, L2::128B unchanged.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global.L2::256B [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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
  // local-reference densities (FP32 pairs, 16-bit storage only): a ring of NPLN
  // planes, each rows y0-2 .. y0+TY+1 over the x window [x0 - 2, x0 + 34)
  static constexpr bool LOCAL = local_ref<ST>();
  static constexpr int RYN = TY + 4, OFFN = 2, WXN = 36, NCHN = 18;
  static constexpr int NPLN = LOCAL ? 4 : 0;
  static constexpr int NPLANE_N = RYN * WXN;  // float2 per ring plane
  // shared-memory carve-up (bytes): NS population stages, the reference-density
  // ring, per-plane row source pointers, row bases, row c^z, then the density / psi rings
  static_assert(STAGE_BYTES % 16 == 0 && NPLANE_N % 2 == 0 && NROW % 2 == 0, "16-byte aligned regions");
  template <int NS> __host__ __device__ static constexpr size_t at_nstage() { return NS * size_t(STAGE_BYTES); }
  template <int NS> __host__ __device__ static constexpr size_t at_rowsrc() { return at_nstage<NS>() + sizeof(float2) * NPLN * NPLANE_N; }
  template <int NS> __host__ __device__ static constexpr size_t at_rowbase() { return at_rowsrc<NS>() + sizeof(void *) * NROW; }
  template <int NS> __host__ __device__ static constexpr size_t at_rowcz() { return at_rowbase<NS>() + sizeof(int64_t) * NROW; }
  template <int NS> __host__ __device__ static constexpr size_t at_ctab() { return at_rowcz<NS>() + sizeof(int) * ((NROW + 3) & ~3); }
  template <int NS> __host__ __device__ static constexpr size_t at_ring() { return at_ctab<NS>() + CTAB_BYTES; }
  // per-thread copy plan (16-bit storage): the NCHUNK 16-byte chunks of a plane's row
  // windows, chunk q = tid + j NT handled by thread tid in round j; entry [j][tid] =
  // (stage byte offset | row << 17, byte offset of the chunk within its source row).
  // It trades the per-chunk index arithmetic for a shared-memory load: faster for
  // 16-bit storage (+3.7 % at 128^3), slower for FP32 (-4 %), so only 16-bit uses it.
  static constexpr bool PLAN = sizeof(ST) == 2;
  static constexpr int NT = 32 * TY;
  static constexpr int NCHUNK = NROW * NCH;
  static constexpr int NPT = (NCHUNK + NT - 1) / NT;
  static constexpr int CTAB_BYTES = PLAN ? NPT * NT * 8 : 0;
  static_assert(STAGE_BYTES <= (1 << 17) && NROW < (1 << 15), "copy-plan entry packing");
};

// Shared memory of one block: the carve-up above, for NS population stages, plus
// the density ring and, with a self coupling (self_on), the psi ring; without
// one the psi ring is never touched and is left out of the launch.
template <class ST, class CT, int TY, int NS>
constexpr size_t staged_smem_bytes(bool self_on = true) {
  using G = StagedGeom<ST, TY>;
  return G::template at_ring<NS>() + sizeof(P2<CT>) * (self_on ? 2 : 1) * G::NPL * G::PLANE;
}

// Sum of the Q staged population pairs arriving at tile position (px, py), in
// direction order (identical to pull_site's order), in natural units; values go to
// v[] (step units, see scaled_units) when V is true.
// With a local reference, nring + nsl[1 - c^z] is the plane of density deviations
// n - nbar of the source plane z - c^z.
template <class ST, class CT, int TY, bool V>
__device__ __forceinline__ P2<CT> staged_sum(const ST *stage, const float2 *nring, const int (&nsl)[3], int px,
                                             int py, P2<CT> scale, P2<CT> inv_scale, P2<CT> *v) {
  using G = StagedGeom<ST, TY>;
  using L = Lattice<kD3Q19>;
  const ST *base = stage + ((py + 1) * G::WX + px + G::OFF) * 2;
  P2<CT> sum = pbc(CT(0));
#pragma unroll
  for (int i = 0; i < G::Q; ++i) {
    P2<CT> g = Codec2<ST, CT>::template load<true>(base + (i * G::RY * G::WX - L::c(i, 0)) * 2, inv_scale);
    if constexpr (G::LOCAL) {
      // density deviation of the source site (x - c_i, y - c_i^y, plane z - c_i^z)
      const float2 ns = nring[nsl[1 - L::c(i, 2)] + (py - L::c(i, 1) + 2) * G::WXN + px + G::OFFN - L::c(i, 0)];
      g = pfma(wpair<kD3Q19, ST, CT>(i, scale), pset(CT(ns.x), CT(ns.y)), g);
    }
    if (V) v[i] = g;
    sum = padd(sum, g);
  }
  return unscale<ST, CT>(sum, inv_scale);
}

// One block's column (bx, by), planes z0 .. zend - 1, of the lattice described by a,
// marched upward or (down) downward; "plane k" below is march position k.
// NS: pipeline stages (2: the copy of plane k + 2 overlaps sum k and collide k - 1;
// 1: the copy of plane k + 1 overlaps collide k - 1 only, for half the stage memory).
// Window x coordinates wrap once: every chunk start lies in [-nx, 2 nx) for nx >= 32.
template <class ST, class CT, int TY, int NS, bool T1>
__device__ __forceinline__ void staged_block(const StepArgs<CT> &a, int bx, int by, int z0, int zend, bool down,
                                             unsigned char *smem_raw) {
  static_assert(NS == 1 || NS == 2, "one or two pipeline stages");
  using G = StagedGeom<ST, TY>;
  using L = Lattice<kD3Q19>;
  constexpr int Q = G::Q;
  constexpr int CQ = carry_size<kD3Q19, T1>();
  constexpr int NT = 32 * TY;
  constexpr int NTASK = (G::NHALO + NT - 1) / NT;  // halo sums per thread and plane
  ST *stage0 = reinterpret_cast<ST *>(smem_raw);                                // [NS][STAGE_ELEMS]
  float2 *nring = reinterpret_cast<float2 *>(smem_raw + G::template at_nstage<NS>());         // [NPLN][RYN][WXN]
  const ST **rowsrc = reinterpret_cast<const ST **>(smem_raw + G::template at_rowsrc<NS>());  // [NROW]
  int64_t *rowbase = reinterpret_cast<int64_t *>(smem_raw + G::template at_rowbase<NS>());    // [NROW]
  int *rowcz = reinterpret_cast<int *>(smem_raw + G::template at_rowcz<NS>());                // [NROW]
  uint2 *ctab = reinterpret_cast<uint2 *>(smem_raw + G::template at_ctab<NS>());              // [NPT][NT]
  P2<CT> *s_dn = reinterpret_cast<P2<CT> *>(smem_raw + G::template at_ring<NS>());            // [NPL][PLANE]
  // [NPL][PLANE]; only read or written under a.self_on (else it aliases s_dn, untouched)
  P2<CT> *s_psi = s_dn + (a.self_on ? G::NPL * G::PLANE : 0);

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t plane_elems = (int64_t)nx * ny;
  const ST *__restrict__ src = static_cast<const ST *>(a.src);
  ST *__restrict__ dst = static_cast<ST *>(a.dst);
  const int x0 = bx * 32, y0 = by * TY;
  const int np = zend - z0 + 2;  // planes z0 - 1 .. zend
  // z of march position k (k = 0 .. np - 1) and of density position m (m = 0 .. np + 1)
  auto zk = [&](int k) { return down ? zend - k : z0 - 1 + k; };
  auto zm = [&](int m) { return down ? zend + 1 - m : z0 - 2 + m; };
  const int own = (ty + 1) * G::SX + (tx + 1);
  const bool valid_xy = (x0 + tx < nx) && (y0 + ty < ny);
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
  // this thread's copy plan (the same chunks every plane; each thread reads back only
  // its own entries, so no barrier is needed): x of the chunk wrapped periodically
  // once here instead of at every copy
#pragma unroll
  for (int j = 0; j < (G::PLAN ? G::NPT : 0); ++j) {
    const int q = tid + j * NT;
    if (q < G::NCHUNK) {
      const int row = q / G::NCH, c = q - row * G::NCH;
      int xs = x0 - G::OFF + c * G::CE;
      xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
      const unsigned soff = unsigned((row * G::WX + c * G::CE) * 2) * unsigned(sizeof(ST));
      ctab[j * NT + tid] = make_uint2(soff | (unsigned(row) << 17), unsigned(xs) * 2u * unsigned(sizeof(ST)));
    }
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
  // copies of the rows in rowsrc into stage s: 16-byte chunks, this thread's part of the
  // copy plan (16-bit storage) or linear over (row, chunk) with the index arithmetic inline
  auto copy_rows = [&](int s) {
    if constexpr (G::PLAN) {
      char *stage = reinterpret_cast<char *>(stage0 + s * G::STAGE_ELEMS);
#pragma unroll
      for (int j = 0; j < G::NPT; ++j) {
        if (j < G::NPT - 1 || tid + j * NT < G::NCHUNK) {
          const uint2 d = ctab[j * NT + tid];
          const char *row = reinterpret_cast<const char *>(rowsrc[d.x >> 17]);
          cp_async16(stage + (d.x & 0x1FFFFu), row + d.y);
        }
      }
    } else {
      ST *stage = stage0 + s * G::STAGE_ELEMS;
      for (int t = tid; t < G::NCHUNK; t += NT) {
        const int row = t / G::NCH, c = t - row * G::NCH;
        int xs = x0 - G::OFF + c * G::CE;
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        cp_async16(stage + (row * G::WX + c * G::CE) * 2, rowsrc[row] + (int64_t)xs * 2);
      }
    }
  };
  // local reference: density position m (z = zm(m)) into ring slot m & 3
  auto copy_nref = [&](int m) {
    if constexpr (G::LOCAL) {
      float2 *dstp = nring + (m & (G::NPLN - 1)) * G::NPLANE_N;
      const int64_t zo = (int64_t)(((zm(m) % nz) + nz) % nz) * ny;  // can wrap more than once for nz < 3
      for (int t = tid; t < G::RYN * G::NCHN; t += NT) {
        const int rr = t / G::NCHN, c = t - rr * G::NCHN;
        int ys = y0 - 2 + rr;
        ys = ((ys % ny) + ny) % ny;
        int xs = x0 - G::OFFN + 2 * c;
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        cp_async16(dstp + rr * G::WXN + 2 * c, a.nsrc + (zo + ys) * nx + xs);
      }
    }
  };
  // commit groups: {plane 0, densities 0-2}, {plane 1, density 3} (two stages), then
  // per body k {plane k + NS, density k + NS + 2}: a group that completes plane p also
  // completes the densities p .. p + 2 its sums read
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    __syncthreads();
    rows_for(wrapz(zk(j)));
    __syncthreads();
    copy_rows(j);
    if (j == 0) {
      copy_nref(0);
      copy_nref(1);
    }
    copy_nref(j + 2);
    cp_async_commit();
  }

  // one plane of the march: sum plane k (the own site's carry into `mine`),
  // then collide plane k - 1 from `prev`
  auto body = [&](int k, P2<CT> (&prev)[CQ], P2<CT> (&mine)[CQ]) {
    const int s = NS == 2 ? (k & 1) : 0;
    const ST *stage = stage0 + s * G::STAGE_ELEMS;
    // density planes of z - 1, z, z + 1 (z = zk(k)): density positions k .. k + 2 (reversed down)
    const int n_lo = (k & 3) * G::NPLANE_N, n_hi = ((k + 2) & 3) * G::NPLANE_N;
    const int nsl[3] = {down ? n_hi : n_lo, ((k + 1) & 3) * G::NPLANE_N, down ? n_lo : n_hi};
    if constexpr (NS == 2)
      cp_async_wait_one();  // all groups but the newest (plane k + 1) are complete: plane k is in
    else
      cp_async_wait_all();
    __syncthreads();  // ... and visible to every thread; the last copy pass is over
    if (k + NS < np) rows_for(wrapz(zk(k + NS)));
    const int slot = k & (G::NPL - 1);
    {
      P2<CT> g[Q];
      const P2<CT> dn = staged_sum<ST, CT, TY, true>(stage, nring, nsl, tx, ty, a.scale, a.inv_scale, g);
      make_carry<kD3Q19, CT, T1>(g, mine);
      s_dn[slot * G::PLANE + own] = dn;
      if (a.self_on) s_psi[slot * G::PLANE + own] = psi_deviation<CT>(dn, a.nbar, a.psibar, a.psi_exp, a.gself);
    }
#pragma unroll
    for (int m = 0; m < NTASK; ++m) {
      if (task_on[m]) {
        const P2<CT> dn =
            staged_sum<ST, CT, TY, false>(stage, nring, nsl, task_px[m], task_py[m], a.scale, a.inv_scale, nullptr);
        s_dn[slot * G::PLANE + task_idx[m]] = dn;
        if (a.self_on) s_psi[slot * G::PLANE + task_idx[m]] = psi_deviation<CT>(dn, a.nbar, a.psibar, a.psi_exp, a.gself);
      }
    }
    __syncthreads();  // stage s and density slot (k + NS + 2) & 3 fully read, ring plane and row pointers written
    if (k + NS < np) copy_rows(s);
    if (k + NS + 2 <= np + 1) copy_nref(k + NS + 2);
    cp_async_commit();  // (possibly empty) group for plane k + NS keeps "newest = plane k + NS"
    if (k >= 2) {
      // ring slots of planes c - 1, c, c + 1 (c = zk(k - 1)): march positions k - 2, k - 1, k
      // (reversed down)
      const int s_lo = (slot + 2) & 3;
      const int sl[3] = {down ? slot : s_lo, (slot + 3) & 3, down ? s_lo : slot};
      const int c = zk(k - 1);
      const int64_t site = (int64_t)gx + (int64_t)nx * (gy + (int64_t)ny * c);
      collide_site<kD3Q19, kE4, ST, CT, TY, T1>(a, prev, s_dn, s_psi, sl, own, valid_xy, dst, site);
    }
  };
  P2<CT> A[CQ], B[CQ];
  int k = 0;
  for (; k + 1 < np; k += 2) {
    body(k, B, A);
    body(k + 1, A, B);
  }
  if (k < np) body(k, B, A);
}

// MINB: resident blocks per SM the register allocation must allow; T1: the
// tau_A = tau_B = 1 form (see carry_size).
template <class ST, class CT, int TY, int NS, int MINB, bool T1>
__global__ void __launch_bounds__(32 * TY, MINB) sc_step_staged(const StepArgs<CT> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int bx, by, z0, zend;
  bool down;
  block_work(a, bx, by, z0, zend, down);
  staged_block<ST, CT, TY, NS, T1>(a, bx, by, z0, zend, down, smem_raw);
}

// Batched form (see sc_step_batched): block b works on items[b] = (lattice, bx,
// by, bz) with the arguments args[lattice], source and destination swapped when
// swap != 0.
template <class ST, class CT, int TY, int NS, int MINB, bool T1>
__global__ void __launch_bounds__(32 * TY, MINB)
    sc_step_staged_batched(const StepArgs<CT> *__restrict__ args, const int4 *__restrict__ items, int swap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the lattice's arguments live in shared memory (read where used, not held in registers)
  __shared__ StepArgs<CT> s_a;
  const int4 it = items[blockIdx.x];
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    StepArgs<CT> a = args[it.x];
    if (swap) {
      const void *t = a.src;
      a.src = a.dst;
      a.dst = const_cast<void *>(t);
      const float2 *u = a.nsrc;
      a.nsrc = a.ndst;
      a.ndst = const_cast<float2 *>(u);
    }
    s_a = a;
  }
  __syncthreads();
  const int z0 = it.w * s_a.tile_z;
  staged_block<ST, CT, TY, NS, T1>(s_a, it.y, it.z, z0, min(z0 + s_a.tile_z, s_a.nz), false, smem_raw);
}

// Grid-wide barrier between the time steps of a persistent launch (all blocks co-resident: the
// launch is cooperative).  Each block arrives once per step on a counter that starts at zero for
// the launch and waits until all gridDim.x blocks have arrived for step t (target (t + 1) gridDim.x).
// The block's stores of the step are made visible device-wide before it arrives; the next step reads
// them through L2 only (cp.async.cg).  The wait is bounded (max_polls polls): false when it ran out.
__device__ __forceinline__ bool grid_step_barrier(unsigned *counter, unsigned target,
                                                  unsigned max_polls = 1u << 20) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
    // polls back off from 64 ns to 4 us (a step takes milliseconds): the waiting blocks keep the L2
    // slice of the counter free for the blocks still working; 2^20 polls take a few seconds
    unsigned spins = 0, pause = 64;
    while (*reinterpret_cast<volatile unsigned *>(counter) < target) {
      if (++spins > max_polls) {
        ok = 0;
        break;
      }
      __nanosleep(pause);
      pause = pause < 4096 ? 2 * pause : pause;
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

// Self-test of the bounded wait: one block waits at the grid barrier for two arrivals of which only
// its own ever comes, so the wait runs out after max_polls polls and, as in a persistent launch, bit 1
// of *err is set.  *counter must be zero.
__global__ void grid_barrier_probe(unsigned *counter, unsigned *err, unsigned max_polls);

// One work item of the persistent launch, compiled as its own function so that its register
// allocation is the one of a single-item block (inlined into the item loop the compiler keeps more
// values live across items); one copy per kernel (MINB), each under that kernel's register limit.
template <class ST, class CT, int TY, int NS, int MINB, bool T1>
__device__ __noinline__ void staged_item(const StepArgs<CT> &a, int bx, int by, int z0, int zend,
                                         unsigned char *smem_raw) {
  staged_block<ST, CT, TY, NS, T1>(a, bx, by, z0, zend, false, smem_raw);
}

// Persistent form of the batched staged step: one cooperative launch runs nsteps time steps of every
// lattice of the batch.  In step t the blocks draw work items (the same list as the per-step launch)
// from the ticket counter counter[1 + t] until the list is exhausted, so that, as with the hardware's
// block dispatch of a per-step launch, a block that finishes early takes the next item; then all meet
// at the grid barrier (counter[0]) before step t + 1.  Step t swaps source and destination when
// (swap0 + t) is odd.  counter[0 .. nsteps] start at zero.  A barrier that runs out sets bit 1 of every
// lattice's status word and ends the launch.
template <class ST, class CT, int TY, int NS, int MINB, bool T1>
__global__ void __launch_bounds__(32 * TY, MINB)
    sc_step_staged_persistent(const StepArgs<CT> *__restrict__ args, const int4 *__restrict__ items, int nitems,
                              int nsteps, int swap0, unsigned *counter, int nlat) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ StepArgs<CT> s_a;
  __shared__ int4 s_it;  // the block's current item; x = -1 when step s_it.y's list is exhausted
  __shared__ int s_t;    // the block's current step
  if (threadIdx.x == 0 && threadIdx.y == 0) s_t = 0;
  for (;;) {
    __syncthreads();  // the previous item is done with the shared arguments, tables and rings
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const int t = s_t;
      const int w = (int)atomicAdd(counter + 1 + t, 1u);
      int4 it = make_int4(-1, t, 0, 0);
      if (w < nitems) {
        it = items[w];
        StepArgs<CT> a = args[it.x];
        if ((swap0 + t) & 1) {
          const void *u = a.src;
          a.src = a.dst;
          a.dst = const_cast<void *>(u);
          const float2 *v = a.nsrc;
          a.nsrc = a.ndst;
          a.ndst = const_cast<float2 *>(v);
        }
        s_a = a;
      }
      s_it = it;
    }
    __syncthreads();
    if (s_it.x >= 0) {
      const int z0 = s_it.w * s_a.tile_z;
      staged_item<ST, CT, TY, NS, MINB, T1>(s_a, s_it.y, s_it.z, z0, min(z0 + s_a.tile_z, s_a.nz), smem_raw);
      continue;
    }
    const int t = s_it.y;  // step t is exhausted: wait for every block, then take step t + 1
    if (t + 1 >= nsteps) return;
    if (!grid_step_barrier(counter, unsigned(t + 1) * gridDim.x)) {
      if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int k = 0; k < nlat; ++k) atomicOr(args[k].err, 2u);
      return;
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) s_t = t + 1;
  }
}

}  // namespace scgb
