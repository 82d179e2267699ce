/*
 * Plain FP64 CPU oracle for the two-component Shan-Chen lattice Boltzmann
 * method of Lulli, Biferale, Falcucci, Sbragaglia and Shan, "Mesoscale
 * Modelling of the Tolman Length in Multi-component Systems" (arXiv:2112.02574).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg and reference arm may
 * load it.  It shares
 * no code, header or table with the CUDA library: every table below is written
 * out here by hand from the paper.
 *
 * Conventions (paper section 2):
 *   - populations f[(J*Q + i)*N + s], J in {0 = A, 1 = B}, s = x + nx*(y + ny*z),
 *     all directions periodic;
 *   - c_s^2 = 1/3;
 *   - lattice velocities xi_i: D3Q19 (paper section 2) or D2Q9 (two-dimensional
 *     analogue, nz = 1);
 *   - forcing stencil: the velocity set's own non-rest vectors with
 *     W(1) = 1/6, W(2) = 1/12 (Eq. sc_force; D2Q9: 1/3, 1/12), or the extended
 *     "E6" set of all integer vectors with |xi|^2 = 1..4 and
 *     W = 2/15, 1/15, 1/60, 1/120.
 * Every step follows Eqs. lbm, omega_i, Guo, feq, u and sc_force in that order:
 *   1. n_J = sum_i f_i,  j_J = sum_i f_i xi_i                      (section 2)
 *   2. psi_J = exp(-1/n_J) or n_J                                  (section 2/4)
 *   3. F_J from Eq. sc_force, +/- stencil pairs summed first
 *   4. n u = sum_J (j_J + F_J/2)                                   (Eq. u)
 *   5. f* = f - (f - f^eq(n_J, u))/tau_J + (1 - 1/(2 tau_J)) F_i^J (Eqs. lbm,
 *      omega_i, Guo, feq)
 *   6. f_i(x + xi_i) <- f*_i(x)                                    (streaming)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t nx, ny, nz;
  int32_t lattice;  /* 0 = D2Q9, 1 = D3Q19 */
  int32_t stencil;  /* 0 = the velocity set's shells (E4), 1 = E6 (D3Q19 only) */
  int32_t psi_self; /* 0: psi = n, 1: psi = exp(-1/n) */
  double tau[2];    /* tau_A, tau_B */
  double G;         /* inter-component coupling of Eq. sc_force */
  double G_self[2]; /* G_AA, G_BB */
} orc_params;

static const double CS2 = 1.0 / 3.0;

/* D3Q19: rest, 6 faces, 12 edges; opposite directions are adjacent (odd, even). */
static const int D3Q19_XI[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
/* D2Q9 in the same spirit (z component zero). */
static const int D2Q9_XI[9][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

/* Lattice weight w_i from |xi_i|^2 (W = w / c_s^2 reproduces the forcing weights
 * printed in section 2: 3 * 1/18 = 1/6 and 3 * 1/36 = 1/12). */
static double lattice_weight(int lattice, int len2) {
  if (lattice == 1) return len2 == 0 ? 1.0 / 3.0 : (len2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  return len2 == 0 ? 4.0 / 9.0 : (len2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
}

int orc_q(int lattice) { return lattice == 1 ? 19 : 9; }

static const int (*velocities(int lattice))[3] { return lattice == 1 ? D3Q19_XI : D2Q9_XI; }

/* ---------------------------------------------------------------- stencil */
/* Half of the forcing stencil: one representative per +/- pair (first
 * non-zero component positive), with its weight W(|xi|^2). */
typedef struct {
  int n;
  int v[16][3];
  double W[16];
} half_stencil;

static double stencil_weight(const orc_params *p, int len2) {
  if (p->stencil == 1) {
    switch (len2) {
      case 1: return 2.0 / 15.0;
      case 2: return 1.0 / 15.0;
      case 3: return 1.0 / 60.0;
      case 4: return 1.0 / 120.0;
      default: return 0.0;
    }
  }
  if (p->lattice == 1) return len2 == 1 ? 1.0 / 6.0 : (len2 == 2 ? 1.0 / 12.0 : 0.0);
  return len2 == 1 ? 1.0 / 3.0 : (len2 == 2 ? 1.0 / 12.0 : 0.0);
}

static void build_half_stencil(const orc_params *p, half_stencil *h) {
  h->n = 0;
  int r = p->stencil == 1 ? 2 : 1;
  int rz = p->lattice == 1 ? r : 0;
  for (int a = -r; a <= r; ++a)
    for (int b = -r; b <= r; ++b)
      for (int c = -rz; c <= rz; ++c) {
        int len2 = a * a + b * b + c * c;
        double W = stencil_weight(p, len2);
        if (len2 == 0 || W == 0.0) continue;
        /* the E4 stencil only holds vectors of the velocity set (|component| <= 1) */
        if (p->stencil == 0 && (abs(a) > 1 || abs(b) > 1 || abs(c) > 1)) continue;
        int first = a != 0 ? a : (b != 0 ? b : c);
        if (first < 0) continue;
        h->v[h->n][0] = a;
        h->v[h->n][1] = b;
        h->v[h->n][2] = c;
        h->W[h->n] = W;
        h->n++;
      }
}

/* Exported for the isotropy pins: full stencil vectors and weights. */
int orc_stencil(const orc_params *p, int *vec /* [n][3] */, double *W) {
  half_stencil h;
  build_half_stencil(p, &h);
  for (int k = 0; k < h.n; ++k) {
    for (int d = 0; d < 3; ++d) {
      vec[(2 * k) * 3 + d] = h.v[k][d];
      vec[(2 * k + 1) * 3 + d] = -h.v[k][d];
    }
    W[2 * k] = W[2 * k + 1] = h.W[k];
  }
  return 2 * h.n;
}

/* ------------------------------------------------------------ indexing */
static inline int wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}
static inline int64_t site_of(const orc_params *p, int x, int y, int z) {
  return (int64_t)wrap(x, p->nx) + (int64_t)p->nx * ((int64_t)wrap(y, p->ny) + (int64_t)p->ny * wrap(z, p->nz));
}
static inline void coords_of(const orc_params *p, int64_t s, int *x, int *y, int *z) {
  *x = (int)(s % p->nx);
  *y = (int)((s / p->nx) % p->ny);
  *z = (int)(s / ((int64_t)p->nx * p->ny));
}
static inline int64_t nsites(const orc_params *p) { return (int64_t)p->nx * p->ny * p->nz; }

/* Pseudopotential of the self-coupling term (section 2 and section 4). */
static inline double psi_of(const orc_params *p, double n) { return p->psi_self == 1 ? exp(-1.0 / n) : n; }

/* ---------------------------------------------------------- initialise */
/* Rest equilibrium f_i = w_i n_J (u = 0). */
void orc_init(const orc_params *p, const double *nA, const double *nB, double *f) {
  const int Q = orc_q(p->lattice);
  const int (*xi)[3] = velocities(p->lattice);
  const int64_t N = nsites(p);
  for (int J = 0; J < 2; ++J) {
    const double *n = J == 0 ? nA : nB;
    for (int i = 0; i < Q; ++i) {
      double w = lattice_weight(p->lattice, xi[i][0] * xi[i][0] + xi[i][1] * xi[i][1] + xi[i][2] * xi[i][2]);
      double *fi = f + ((int64_t)J * Q + i) * N;
#pragma omp parallel for schedule(static)
      for (int64_t s = 0; s < N; ++s) fi[s] = w * n[s];
    }
  }
}

/* ------------------------------------------------------------- moments */
/* n_J = sum_i f_i^J  (section 2). */
void orc_density(const orc_params *p, const double *f, double *nA, double *nB) {
  const int Q = orc_q(p->lattice);
  const int64_t N = nsites(p);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < N; ++s) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < Q; ++i) {
      a += f[(int64_t)i * N + s];
      b += f[((int64_t)Q + i) * N + s];
    }
    nA[s] = a;
    nB[s] = b;
  }
}

/* Shan-Chen force of Eq. sc_force at site s, both components.
 *   F_A = -G c_s^2 n_A sum_a W n_B(x+xi_a) xi_a - G_AA c_s^2 psi_A sum_a W psi_A(x+xi_a) xi_a
 *   F_B = (A <-> B)
 * Each sum runs over +/- pairs: W xi_a [g(x + xi_a) - g(x - xi_a)]. */
static void sc_force_at(const orc_params *p, const half_stencil *h, const double *nA, const double *nB,
                        const double *psiA, const double *psiB, int64_t s, double FA[3], double FB[3]) {
  int x, y, z;
  coords_of(p, s, &x, &y, &z);
  double SA[3] = {0, 0, 0}, SB[3] = {0, 0, 0}, TA[3] = {0, 0, 0}, TB[3] = {0, 0, 0};
  for (int k = 0; k < h->n; ++k) {
    const int *v = h->v[k];
    int64_t sp = site_of(p, x + v[0], y + v[1], z + v[2]);
    int64_t sm = site_of(p, x - v[0], y - v[1], z - v[2]);
    double dA = nA[sp] - nA[sm], dB = nB[sp] - nB[sm];
    double dpA = psiA[sp] - psiA[sm], dpB = psiB[sp] - psiB[sm];
    for (int m = 0; m < 3; ++m) {
      SA[m] += h->W[k] * v[m] * dA;
      SB[m] += h->W[k] * v[m] * dB;
      TA[m] += h->W[k] * v[m] * dpA;
      TB[m] += h->W[k] * v[m] * dpB;
    }
  }
  for (int m = 0; m < 3; ++m) {
    FA[m] = -p->G * CS2 * nA[s] * SB[m] - p->G_self[0] * CS2 * psiA[s] * TA[m];
    FB[m] = -p->G * CS2 * nB[s] * SA[m] - p->G_self[1] * CS2 * psiB[s] * TB[m];
  }
}

static void psi_field(const orc_params *p, const double *n, double *psi) {
  const int64_t N = nsites(p);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < N; ++s) psi[s] = psi_of(p, n[s]);
}

/* Force field F_A, F_B ([3][N] each) from density fields. */
void orc_force(const orc_params *p, const double *nA, const double *nB, double *FA, double *FB) {
  const int64_t N = nsites(p);
  half_stencil h;
  build_half_stencil(p, &h);
  double *psiA = malloc(sizeof(double) * N), *psiB = malloc(sizeof(double) * N);
  psi_field(p, nA, psiA);
  psi_field(p, nB, psiB);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < N; ++s) {
    double a[3], b[3];
    sc_force_at(p, &h, nA, nB, psiA, psiB, s, a, b);
    for (int m = 0; m < 3; ++m) {
      FA[m * N + s] = a[m];
      FB[m * N + s] = b[m];
    }
  }
  free(psiA);
  free(psiB);
}

/* Common velocity of Eq. u at site s: n u = sum_J (j_J + F_J / 2). */
static void velocity_at(const orc_params *p, const double *f, int64_t s, double nA, double nB, const double FA[3],
                        const double FB[3], double u[3]) {
  const int Q = orc_q(p->lattice);
  const int (*xi)[3] = velocities(p->lattice);
  const int64_t N = nsites(p);
  double jA[3] = {0, 0, 0}, jB[3] = {0, 0, 0};
  for (int i = 0; i < Q; ++i) {
    double a = f[(int64_t)i * N + s], b = f[((int64_t)Q + i) * N + s];
    for (int m = 0; m < 3; ++m) {
      jA[m] += a * xi[i][m];
      jB[m] += b * xi[i][m];
    }
  }
  for (int m = 0; m < 3; ++m) u[m] = ((jA[m] + 0.5 * FA[m]) + (jB[m] + 0.5 * FB[m])) / (nA + nB);
}

/* n_A, n_B and the common velocity u ([3][N], may be NULL) of state f. */
void orc_moments(const orc_params *p, const double *f, double *nA, double *nB, double *u) {
  const int64_t N = nsites(p);
  orc_density(p, f, nA, nB);
  if (!u) return;
  double *FA = malloc(sizeof(double) * 3 * N), *FB = malloc(sizeof(double) * 3 * N);
  orc_force(p, nA, nB, FA, FB);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < N; ++s) {
    double a[3] = {FA[s], FA[N + s], FA[2 * N + s]}, b[3] = {FB[s], FB[N + s], FB[2 * N + s]}, uu[3];
    velocity_at(p, f, s, nA[s], nB[s], a, b, uu);
    for (int m = 0; m < 3; ++m) u[m * N + s] = uu[m];
  }
  free(FA);
  free(FB);
}

/* BGK collision with Guo forcing at one site, component J (Eqs. lbm, omega_i,
 * Guo, feq): out[i] = f_i - (f_i - f_i^eq)/tau + (1 - 1/(2 tau)) F_i. */
static void collide_at(const orc_params *p, int J, const double *fs /* Q values */, double n, const double u[3],
                       const double F[3], double *out) {
  const int Q = orc_q(p->lattice);
  const int (*xi)[3] = velocities(p->lattice);
  const double tau = p->tau[J];
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  for (int i = 0; i < Q; ++i) {
    double w = lattice_weight(p->lattice, xi[i][0] * xi[i][0] + xi[i][1] * xi[i][1] + xi[i][2] * xi[i][2]);
    double xu = xi[i][0] * u[0] + xi[i][1] * u[1] + xi[i][2] * u[2];
    double xF = xi[i][0] * F[0] + xi[i][1] * F[1] + xi[i][2] * F[2];
    double feq = n * w * (1.0 + xu / CS2 + (xu * xu - CS2 * uu) / (2.0 * CS2 * CS2));
    double Fi = w * (xF / CS2 + (xu * xF - CS2 * uF) / (CS2 * CS2));
    out[i] = fs[i] - (fs[i] - feq) / tau + (1.0 - 1.0 / (2.0 * tau)) * Fi;
  }
}

/* Post-collision populations of both components at site s, given density and
 * pseudopotential fields of the current state.  out: [2][Q]. */
static void post_collision_at(const orc_params *p, const half_stencil *h, const double *f, const double *nA,
                              const double *nB, const double *psiA, const double *psiB, int64_t s, double *out) {
  const int Q = orc_q(p->lattice);
  const int64_t N = nsites(p);
  double FA[3], FB[3], u[3], fs[19];
  sc_force_at(p, h, nA, nB, psiA, psiB, s, FA, FB);
  velocity_at(p, f, s, nA[s], nB[s], FA, FB, u);
  for (int J = 0; J < 2; ++J) {
    for (int i = 0; i < Q; ++i) fs[i] = f[((int64_t)J * Q + i) * N + s];
    collide_at(p, J, fs, J == 0 ? nA[s] : nB[s], u, J == 0 ? FA : FB, out + J * Q);
  }
}

/* nsteps full time steps; f is updated in place (tmp: same size as f). */
void orc_step(const orc_params *p, double *f, double *tmp, int nsteps) {
  const int Q = orc_q(p->lattice);
  const int (*xi)[3] = velocities(p->lattice);
  const int64_t N = nsites(p);
  half_stencil h;
  build_half_stencil(p, &h);
  double *nA = malloc(sizeof(double) * N), *nB = malloc(sizeof(double) * N);
  double *psiA = malloc(sizeof(double) * N), *psiB = malloc(sizeof(double) * N);
  for (int t = 0; t < nsteps; ++t) {
    orc_density(p, f, nA, nB);
    psi_field(p, nA, psiA);
    psi_field(p, nB, psiB);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
      double post[38];
      post_collision_at(p, &h, f, nA, nB, psiA, psiB, s, post);
      int x, y, z;
      coords_of(p, s, &x, &y, &z);
      for (int J = 0; J < 2; ++J)
        for (int i = 0; i < Q; ++i)
          tmp[((int64_t)J * Q + i) * N + site_of(p, x + xi[i][0], y + xi[i][1], z + xi[i][2])] = post[J * Q + i];
    }
    memcpy(f, tmp, sizeof(double) * 2 * Q * N);
  }
  free(nA);
  free(nB);
  free(psiA);
  free(psiB);
}

/* One time step evaluated only at the listed sites: out[(J*Q + i)*nsel + k] is
 * f_i^J(site_k, t + 1) = f*_i^J(site_k - xi_i, t).  Each needed upstream site is
 * collided from the full state f. */
void orc_step_sites(const orc_params *p, const double *f, const int64_t *sel, int64_t nsel, double *out) {
  const int Q = orc_q(p->lattice);
  const int (*xi)[3] = velocities(p->lattice);
  const int64_t N = nsites(p);
  half_stencil h;
  build_half_stencil(p, &h);
  double *nA = malloc(sizeof(double) * N), *nB = malloc(sizeof(double) * N);
  double *psiA = malloc(sizeof(double) * N), *psiB = malloc(sizeof(double) * N);
  orc_density(p, f, nA, nB);
  psi_field(p, nA, psiA);
  psi_field(p, nB, psiB);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < nsel; ++k) {
    int x, y, z;
    coords_of(p, sel[k], &x, &y, &z);
    for (int i = 0; i < Q; ++i) {
      double post[38];
      int64_t up = site_of(p, x - xi[i][0], y - xi[i][1], z - xi[i][2]);
      post_collision_at(p, &h, f, nA, nB, psiA, psiB, up, post);
      out[((int64_t)0 * Q + i) * nsel + k] = post[i];
      out[((int64_t)1 * Q + i) * nsel + k] = post[Q + i];
    }
  }
  free(nA);
  free(nB);
  free(psiA);
  free(psiB);
}

/* Totals for the conservation pins: mass[2] = sum_x n_J, mom[3] = sum_x sum_J sum_i f_i xi_i. */
void orc_totals(const orc_params *p, const double *f, double *mass, double *mom) {
  const int Q = orc_q(p->lattice);
  const int (*xi)[3] = velocities(p->lattice);
  const int64_t N = nsites(p);
  for (int J = 0; J < 2; ++J) {
    double m = 0.0;
    for (int i = 0; i < Q; ++i) {
      const double *fi = f + ((int64_t)J * Q + i) * N;
      /* Kahan-compensated sum keeps the pin at round-off level */
      double c = 0.0;
      for (int64_t s = 0; s < N; ++s) {
        double y = fi[s] - c, t = m + y;
        c = (t - m) - y;
        m = t;
      }
    }
    mass[J] = m;
  }
  for (int m = 0; m < 3; ++m) {
    double acc = 0.0, c = 0.0;
    for (int J = 0; J < 2; ++J)
      for (int i = 0; i < Q; ++i) {
        if (xi[i][m] == 0) continue;
        const double *fi = f + ((int64_t)J * Q + i) * N;
        for (int64_t s = 0; s < N; ++s) {
          double y = xi[i][m] * fi[s] - c, t = acc + y;
          c = (t - acc) - y;
          acc = t;
        }
      }
    mom[m] = acc;
  }
}

/* ---------------------------------------------------- pressure tensor */
/* Bulk pressure of Eq. bulkp (e_2 = 1 for every stencil used here). */
double orc_bulk_pressure(const orc_params *p, double nA, double nB) {
  const double e2 = 1.0;
  double psiA = psi_of(p, nA), psiB = psi_of(p, nB);
  return (nA + nB) * CS2 + p->G * CS2 * e2 * nA * nB + 0.5 * p->G_self[0] * CS2 * e2 * psiA * psiA +
         0.5 * p->G_self[1] * CS2 * e2 * psiB * psiB;
}

/* Lattice pressure tensor of Eq. sm:pt at site s; P = {xx, yy, zz, xy, xz, yz}.
 * The stencil sums run over the full stencil (+xi and -xi both). */
static void ptensor_at(const orc_params *p, const half_stencil *h, const double *nA, const double *nB,
                       const double *psiA, const double *psiB, int64_t s, double P[6]) {
  static const int MU[6] = {0, 1, 2, 0, 0, 1}, NU[6] = {0, 1, 2, 1, 2, 2};
  int x, y, z;
  coords_of(p, s, &x, &y, &z);
  double cross_A[6] = {0}, cross_B[6] = {0}, self_A[6] = {0}, self_B[6] = {0};
  for (int k = 0; k < h->n; ++k)
    for (int sgn = 1; sgn >= -1; sgn -= 2) {
      int v[3] = {sgn * h->v[k][0], sgn * h->v[k][1], sgn * h->v[k][2]};
      int64_t sn = site_of(p, x + v[0], y + v[1], z + v[2]);
      for (int c = 0; c < 6; ++c) {
        double xx = h->W[k] * v[MU[c]] * v[NU[c]];
        cross_A[c] += xx * nB[sn]; /* n_A(x) sum W n_B(x + xi) xi xi */
        cross_B[c] += xx * nA[sn]; /* n_B(x) sum W n_A(x + xi) xi xi */
        self_A[c] += xx * psiA[sn];
        self_B[c] += xx * psiB[sn];
      }
    }
  for (int c = 0; c < 6; ++c) {
    double ideal = c < 3 ? (nA[s] + nB[s]) * CS2 : 0.0;
    P[c] = ideal + 0.5 * p->G * CS2 * nA[s] * cross_A[c] + 0.5 * p->G * CS2 * nB[s] * cross_B[c] +
           0.5 * p->G_self[0] * CS2 * psiA[s] * self_A[c] + 0.5 * p->G_self[1] * CS2 * psiB[s] * self_B[c];
  }
}

/* Full tensor field, P[c*N + s], c in {xx, yy, zz, xy, xz, yz}. */
void orc_pressure_tensor(const orc_params *p, const double *nA, const double *nB, double *P) {
  const int64_t N = nsites(p);
  half_stencil h;
  build_half_stencil(p, &h);
  double *psiA = malloc(sizeof(double) * N), *psiB = malloc(sizeof(double) * N);
  psi_field(p, nA, psiA);
  psi_field(p, nB, psiB);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < N; ++s) {
    double t[6];
    ptensor_at(p, &h, nA, nB, psiA, psiB, s, t);
    for (int c = 0; c < 6; ++c) P[c * N + s] = t[c];
  }
  free(psiA);
  free(psiB);
}

/* ------------------------------------------------------------ profiles */
/* Output rows [nbins][6] = (mean coordinate, P_N, P_T, n_A, n_B, count); empty
 * bins are all zero.  kind 0: radial shells of width bin_width around centre
 * (minimum image), P_N = rhat.P.rhat, P_T = (tr P - P_N)/(d - 1), and at r = 0
 * P_N = P_T = tr P / d (decomposition Eq. pt_projection).  kind 1: planes of
 * constant z, P_N = <P^zz>, P_T = <(P^xx + P^yy)/2> (flat interface, section 4).
 * kind 2: the x axis through the centre node, P_N = P^xx, P_T = P^yy (section 3). */
void orc_profile(const orc_params *p, const double *nA, const double *nB, int kind, const double centre[3],
                 double bin_width, int nbins, double *out) {
  const int64_t N = nsites(p);
  const int dim = (p->lattice == 1 && p->nz > 1) ? 3 : 2;
  double *P = malloc(sizeof(double) * 6 * N);
  orc_pressure_tensor(p, nA, nB, P);
  double *acc = calloc((size_t)nbins * 6, sizeof(double));
  if (kind == 0) {
    for (int64_t s = 0; s < N; ++s) {
      int x, y, z;
      coords_of(p, s, &x, &y, &z);
      int c[3] = {x, y, z}, L[3] = {p->nx, p->ny, p->nz};
      double d[3];
      for (int m = 0; m < 3; ++m) {
        double dd = c[m] - centre[m];
        dd -= L[m] * floor(dd / L[m] + 0.5); /* minimum image, in [-L/2, L/2) */
        d[m] = dd;
      }
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      int k = (int)floor(r / bin_width);
      if (k >= nbins) continue;
      double Pxx = P[s], Pyy = P[N + s], Pzz = P[2 * N + s], Pxy = P[3 * N + s], Pxz = P[4 * N + s],
             Pyz = P[5 * N + s];
      double tr = dim == 3 ? Pxx + Pyy + Pzz : Pxx + Pyy;
      double PN, PT;
      if (r == 0.0) {
        PN = PT = tr / dim;
      } else {
        double e[3] = {d[0] / r, d[1] / r, d[2] / r};
        PN = e[0] * e[0] * Pxx + e[1] * e[1] * Pyy + e[2] * e[2] * Pzz + 2.0 * e[0] * e[1] * Pxy +
             2.0 * e[0] * e[2] * Pxz + 2.0 * e[1] * e[2] * Pyz;
        PT = (tr - PN) / (dim - 1);
      }
      double *row = acc + 6 * k;
      row[0] += r;
      row[1] += PN;
      row[2] += PT;
      row[3] += nA[s];
      row[4] += nB[s];
      row[5] += 1.0;
    }
  } else if (kind == 1) {
    for (int64_t s = 0; s < N; ++s) {
      int x, y, z;
      coords_of(p, s, &x, &y, &z);
      if (z >= nbins) continue;
      double *row = acc + 6 * z;
      row[0] += z;
      row[1] += P[2 * N + s];
      row[2] += 0.5 * (P[s] + P[N + s]);
      row[3] += nA[s];
      row[4] += nB[s];
      row[5] += 1.0;
    }
  } else {
    int cx = (int)floor(centre[0] + 0.5), cy = (int)floor(centre[1] + 0.5), cz = (int)floor(centre[2] + 0.5);
    for (int k = 0; k < nbins; ++k) {
      int64_t s = site_of(p, cx + k, cy, cz);
      double *row = acc + 6 * k;
      row[0] = k;
      row[1] = P[s];
      row[2] = P[N + s];
      row[3] = nA[s];
      row[4] = nB[s];
      row[5] = 1.0;
    }
  }
  for (int k = 0; k < nbins; ++k) {
    double *row = acc + 6 * k;
    double cnt = row[5];
    out[6 * k + 5] = cnt;
    for (int c = 0; c < 5; ++c) out[6 * k + c] = cnt > 0 ? row[c] / cnt : 0.0;
  }
  free(acc);
  free(P);
}

/* The velocity set and its weights, for the isotropy pins. */
int orc_velocity_set(int lattice, int *xi_out /* [Q][3] */, double *w_out) {
  const int Q = orc_q(lattice);
  const int (*xi)[3] = velocities(lattice);
  for (int i = 0; i < Q; ++i) {
    for (int d = 0; d < 3; ++d) xi_out[3 * i + d] = xi[i][d];
    w_out[i] = lattice_weight(lattice, xi[i][0] * xi[i][0] + xi[i][1] * xi[i][1] + xi[i][2] * xi[i][2]);
  }
  return Q;
}

/* Threads the OpenMP loops above use. */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(void) { return omp_get_max_threads(); }
#else
int orc_threads(void) { return 1; }
#endif
