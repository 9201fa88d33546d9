/*
 * rbe_oracle.c -- plain FP64 CPU oracle for the improved random batch Ewald force path
 * of RBMD 2.0 (arXiv 2609.02694, Sec. 2.1, Eqs. potential .. F_corr).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg, never by the product library. Shares no code with it.
 *
 * Every function follows the definition it cites, term by term, in FP64, summing in
 * ascending particle id and ascending mode index. Build with -ffp-contract=off so that
 * no multiply-add is fused. OpenMP, where present, only splits loops whose iterations
 * write disjoint outputs; every sum keeps its serial order.
 *
 * Parity is pinned (tests/test_oracle_*.py) by: Philox known-answer vectors; the Poisson
 * summation closed form of the sampling normaliser and a chi-square test of the draws;
 * the NaCl Madelung constant; brute-force image sums; alpha-invariance; finite
 * differences of every energy; zero net RBE force; unbiasedness of RBE and RBL over
 * seeds; the exact limits of RBL; the LJ zero-force distance.
 */
#include "rbe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#define TWO32 4294967296.0

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ---------------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4): ten rounds of two 32x32->64 products
 * with multipliers 0xD2511F53 and 0xCD9E8D57, the key bumped between rounds by the Weyl
 * constants 0x9E3779B9 and 0xBB67AE85. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ---------------------------------------------------------------------------------- */
/* Sampling density of Eq. F_long_RBE: P(k) ~ exp(-k^2/(4 alpha)) on K \ {0}. With
 * k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z) the weight is a product over axes, so each axis is
 * an independent 1-D discrete Gaussian, truncated where its weight drops below 2^-53. */
int orc_kdim_M(double L, double alpha) {
  return (int)ceil(L * sqrt(4.0 * alpha * 53.0 * log(2.0)) / (2.0 * M_PI));
}

static double kdim_weight(int mi, double L, double alpha) {
  double km = 2.0 * M_PI * (double)mi / L;
  return exp(-(km * km) / (4.0 * alpha));
}

int orc_kdim_table(double L, double alpha, int M, uint64_t *T, double *Z) {
  if (!(L > 0) || !(alpha > 0) || M < 0) return -1;
  int n = 2 * M + 1;
  double z = 0.0;
  for (int i = 0; i < n; ++i) z += kdim_weight(i - M, L, alpha);
  double acc = 0.0;
  for (int i = 0; i < n; ++i) {
    acc += kdim_weight(i - M, L, alpha);
    T[i] = (uint64_t)floor(acc / z * TWO32);
  }
  T[n - 1] = (uint64_t)1 << 32;
  *Z = z;
  return 0;
}

int orc_sample_k(uint64_t seed, uint64_t step, uint32_t replica, const double box[3],
                 double alpha, int P, int32_t *m, double *S) {
  if (P <= 0 || !(alpha > 0)) return -1;
  int M[3];
  uint64_t *T[3];
  double Z[3];
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0)) return -1;
    M[d] = orc_kdim_M(box[d], alpha);
    T[d] = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * M[d] + 1));
    orc_kdim_table(box[d], alpha, M[d], T[d], &Z[d]);
  }
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ replica};
  int rc = 0;
  for (int l = 0; l < P && rc == 0; ++l) {
    int done = 0;
    for (uint32_t attempt = 0; attempt < 64 && !done; ++attempt) {
      uint32_t ctr[4] = {(uint32_t)l, attempt, (uint32_t)step, 0u};
      uint32_t w[4];
      orc_philox4x32_10(ctr, key, w);
      int md[3];
      for (int d = 0; d < 3; ++d) {
        int i = 0; /* smallest index with w_d < T_d[i] (linear scan) */
        while ((uint64_t)w[d] >= T[d][i]) ++i;
        md[d] = i - M[d];
      }
      if (md[0] != 0 || md[1] != 0 || md[2] != 0) {
        for (int d = 0; d < 3; ++d) m[3 * l + d] = md[d];
        done = 1;
      }
    }
    if (!done) rc = -2;
  }
  *S = Z[0] * Z[1] * Z[2] - 1.0;
  for (int d = 0; d < 3; ++d) free(T[d]);
  return rc;
}

/* ---------------------------------------------------------------------------------- */
static void kvec(const int32_t *m, const double box[3], double k[3]) {
  for (int d = 0; d < 3; ++d) k[d] = 2.0 * M_PI * (double)m[d] / box[d];
}

static void position(const uint32_t *s, const double box[3], double r[3]) {
  for (int d = 0; d < 3; ++d) r[d] = (double)s[d] * (box[d] / TWO32);
}

/* rho(k) = sum_j q_j exp(i k . r_j), Eq. U_Coul_Fourier. */
int orc_rho(int64_t N, const uint32_t *s, const double *q, const double box[3], int P,
            const int32_t *m, double *rho) {
  if (N < 0 || P < 0) return -1;
#pragma omp parallel for schedule(static)
  for (int l = 0; l < P; ++l) {
    double k[3];
    kvec(&m[3 * l], box, k);
    double re = 0.0, im = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      double r[3];
      position(&s[3 * j], box, r);
      double kr = k[0] * r[0] + k[1] * r[1] + k[2] * r[2];
      re += q[j] * cos(kr);
      im += q[j] * sin(kr);
    }
    rho[2 * l] = re;
    rho[2 * l + 1] = im;
  }
  return 0;
}

/* Eq. F_long_RBE (with the minus sign of Eq. F_i):
 *   F_i = -(S/P) sum_l 4 pi C q_i k_l / (V k_l^2) Im(exp(-i k_l.r_i) rho_l),
 * Im(exp(-i theta)(a + i b)) = b cos theta - a sin theta. */
int orc_rbe_kspace(int64_t N, const uint32_t *s, const double *q, const double box[3],
                   double alpha, double C, int P, const int32_t *m, double S,
                   double *F, double *U, double *W) {
  if (N < 0 || P <= 0) return -1;
  double V = box[0] * box[1] * box[2];
  double *rho = (double *)malloc(sizeof(double) * 2 * (size_t)P);
  orc_rho(N, s, q, box, P, m, rho);
  double u = 0.0, w = 0.0;
  for (int l = 0; l < P; ++l) {
    double k[3];
    kvec(&m[3 * l], box, k);
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    double rho2 = rho[2 * l] * rho[2 * l] + rho[2 * l + 1] * rho[2 * l + 1];
    double El = (S / (double)P) * 2.0 * M_PI * C * rho2 / (V * k2);
    u += El;
    w += El * (1.0 - k2 / (2.0 * alpha));
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    double r[3], f[3] = {0.0, 0.0, 0.0};
    position(&s[3 * i], box, r);
    for (int l = 0; l < P; ++l) {
      double k[3];
      kvec(&m[3 * l], box, k);
      double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
      double kr = k[0] * r[0] + k[1] * r[1] + k[2] * r[2];
      double im = rho[2 * l + 1] * cos(kr) - rho[2 * l] * sin(kr);
      double c = (S / (double)P) * 4.0 * M_PI * C * q[i] / (V * k2);
      for (int d = 0; d < 3; ++d) f[d] -= c * k[d] * im;
    }
    for (int d = 0; d < 3; ++d) F[3 * i + d] = f[d];
  }
  free(rho);
  if (U) *U = u;
  if (W) *W = w;
  return 0;
}

/* Full Ewald k-space sum (Eqs. U_Coul_Fourier and F_i) over every m != 0 with
 * |m_d| <= M_d, where M_d is the half-width at which exp(-k^2/4 alpha) < 2^-53. */
/* Eqs. U_Coul_Fourier and F_i summed over the P modes of mlist (frees mlist). */
static int ewald_over_modes(int64_t N, const uint32_t *s, const double *q, const double box[3],
                            double alpha, double C, int64_t P, int32_t *mlist, double *F,
                            double *U, double *W);

int orc_ewald_kspace(int64_t N, const uint32_t *s, const double *q, const double box[3],
                     double alpha, double C, double *F, double *U, double *W) {
  if (N < 0) return -1;
  int M[3];
  for (int d = 0; d < 3; ++d) M[d] = orc_kdim_M(box[d], alpha);
  int64_t nm = (int64_t)(2 * M[0] + 1) * (2 * M[1] + 1) * (2 * M[2] + 1);
  int32_t *mlist = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nm);
  int64_t P = 0;
  for (int mz = -M[2]; mz <= M[2]; ++mz)
    for (int my = -M[1]; my <= M[1]; ++my)
      for (int mx = -M[0]; mx <= M[0]; ++mx) {
        if (mx == 0 && my == 0 && mz == 0) continue;
        mlist[3 * P] = mx; mlist[3 * P + 1] = my; mlist[3 * P + 2] = mz;
        ++P;
      }
  return ewald_over_modes(N, s, q, box, alpha, C, P, mlist, F, U, W);
}

/* The same sum truncated at a stated accuracy, the way Ewald and mesh solvers are run in
 * practice (the paper's own reference runs use a mesh solver at a 1e-4 tolerance, Sec. 3.1):
 * only the modes k != 0 whose weight exp(-k^2 / 4 alpha) is at least tol enter, a sphere
 * |k|^2 <= 4 alpha ln(1/tol), in the same ascending (m_z, m_y, m_x) order. */
int orc_ewald_kspace_tol(int64_t N, const uint32_t *s, const double *q, const double box[3],
                         double alpha, double C, double tol, double *F, double *U, double *W) {
  if (N < 0 || !(tol > 0.0) || !(tol < 1.0)) return -1;
  const double k2max = 4.0 * alpha * log(1.0 / tol);
  int M[3];
  for (int d = 0; d < 3; ++d) M[d] = (int)ceil(box[d] * sqrt(k2max) / (2.0 * M_PI));
  int64_t nm = (int64_t)(2 * M[0] + 1) * (2 * M[1] + 1) * (2 * M[2] + 1);
  int32_t *mlist = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nm);
  int64_t P = 0;
  for (int mz = -M[2]; mz <= M[2]; ++mz)
    for (int my = -M[1]; my <= M[1]; ++my)
      for (int mx = -M[0]; mx <= M[0]; ++mx) {
        if (mx == 0 && my == 0 && mz == 0) continue;
        const int32_t m[3] = {mx, my, mz};
        double k[3];
        kvec(m, box, k);
        if (k[0] * k[0] + k[1] * k[1] + k[2] * k[2] > k2max) continue;
        mlist[3 * P] = mx; mlist[3 * P + 1] = my; mlist[3 * P + 2] = mz;
        ++P;
      }
  return ewald_over_modes(N, s, q, box, alpha, C, P, mlist, F, U, W);
}

static int ewald_over_modes(int64_t N, const uint32_t *s, const double *q, const double box[3],
                            double alpha, double C, int64_t P, int32_t *mlist, double *F,
                            double *U, double *W) {
  double V = box[0] * box[1] * box[2];
  double *rho = (double *)malloc(sizeof(double) * 2 * (size_t)P);
  double *g = (double *)malloc(sizeof(double) * (size_t)P); /* exp(-k^2/4a)/k^2 */
  orc_rho(N, s, q, box, (int)P, mlist, rho);
  double u = 0.0, w = 0.0;
  for (int64_t l = 0; l < P; ++l) {
    double k[3];
    kvec(&mlist[3 * l], box, k);
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    g[l] = exp(-k2 / (4.0 * alpha)) / k2;
    double rho2 = rho[2 * l] * rho[2 * l] + rho[2 * l + 1] * rho[2 * l + 1];
    double El = 2.0 * M_PI * C / V * rho2 * g[l];
    u += El;
    w += El * (1.0 - k2 / (2.0 * alpha));
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    double r[3], f[3] = {0.0, 0.0, 0.0};
    position(&s[3 * i], box, r);
    for (int64_t l = 0; l < P; ++l) {
      double k[3];
      kvec(&mlist[3 * l], box, k);
      double kr = k[0] * r[0] + k[1] * r[1] + k[2] * r[2];
      double im = rho[2 * l + 1] * cos(kr) - rho[2 * l] * sin(kr);
      double c = 4.0 * M_PI * C * q[i] / V * g[l];
      for (int d = 0; d < 3; ++d) f[d] -= c * k[d] * im;
    }
    for (int d = 0; d < 3; ++d) F[3 * i + d] = f[d];
  }
  free(mlist); free(rho); free(g);
  if (U) *U = u;
  if (W) *W = w;
  return 0;
}

double orc_self_energy(int64_t N, const double *q, double alpha, double C) {
  double sq = 0.0;
  for (int64_t i = 0; i < N; ++i) sq += q[i] * q[i];
  return C * sqrt(alpha / M_PI) * sq;
}

/* ---------------------------------------------------------------------------------- */
/* Minimum image (Sec. 2.1): on the 2^-32 grid the closest periodic image of the
 * separation is the two's-complement difference of the fractional coordinates. */
double orc_min_image_r2(const uint32_t *si, const uint32_t *sj, const double box[3],
                        double d[3]) {
  for (int k = 0; k < 3; ++k)
    d[k] = (double)(int32_t)(si[k] - sj[k]) * (box[k] / TWO32);
  return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

/* One pair (Eqs. F_i, G_short, LJ): force factor g with F_ij = g (r_i - r_j), the two
 * energies and the two virial terms. */
static void pair_terms(double r2, double qq, double alpha, double C, double eps,
                       double sig, double *g, double *ucoul, double *ulj, double *wcoul,
                       double *wlj) {
  double r = sqrt(r2);
  double gc = 0.0, uc = 0.0;
  if (qq != 0.0) {
    double sa = sqrt(alpha);
    double G = erfc(sa * r) / (r2 * r) + 2.0 * sa * exp(-alpha * r2) / (sqrt(M_PI) * r2);
    gc = C * qq * G;
    uc = C * qq * erfc(sa * r) / r;
  }
  double gl = 0.0, ul = 0.0;
  if (eps != 0.0) {
    double sr2 = sig * sig / r2;
    double sr6 = sr2 * sr2 * sr2;
    double sr12 = sr6 * sr6;
    gl = 24.0 * eps * (2.0 * sr12 - sr6) / r2; /* = 24 eps (2 sig^12/r^14 - sig^6/r^8) */
    ul = 4.0 * eps * (sr12 - sr6);
  }
  *g = gc + gl;
  *ucoul = uc;
  *ulj = ul;
  *wcoul = gc * r2;
  *wlj = gl * r2;
}

int orc_real_space(int64_t N, const uint32_t *s, const double *q, const int32_t *type,
                   const double box[3], double alpha, double rc, double C, int ntypes,
                   const double *eps, const double *sig, const int64_t *i_list,
                   int64_t n_list, double *F, double *U_real, double *U_lj,
                   double *W_real, double *W_lj, int32_t *nbr_count) {
  if (N < 0 || ntypes < 1 || !(rc > 0)) return -1;
  for (int d = 0; d < 3; ++d)
    if (!(2.0 * rc < box[d])) return -3; /* the minimum image must be unique */
  int64_t n_eval = i_list ? n_list : N;
  double rc2 = rc * rc;
  double *ui = (double *)calloc((size_t)n_eval * 4, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < n_eval; ++t) {
    int64_t i = i_list ? i_list[t] : t;
    double f[3] = {0.0, 0.0, 0.0}, uc = 0.0, ul = 0.0, wc = 0.0, wl = 0.0;
    int32_t cnt = 0;
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      double d[3];
      double r2 = orc_min_image_r2(&s[3 * i], &s[3 * j], box, d);
      if (!(r2 <= rc2)) continue;
      ++cnt;
      int pt = type[i] * ntypes + type[j];
      double g, a, b, c, e;
      pair_terms(r2, q[i] * q[j], alpha, C, eps[pt], sig[pt], &g, &a, &b, &c, &e);
      for (int k = 0; k < 3; ++k) f[k] += g * d[k];
      uc += a; ul += b; wc += c; wl += e;
    }
    for (int k = 0; k < 3; ++k) F[3 * i + k] = f[k];
    ui[4 * t] = uc; ui[4 * t + 1] = ul; ui[4 * t + 2] = wc; ui[4 * t + 3] = wl;
    if (nbr_count) nbr_count[i] = cnt;
  }
  double sums[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t t = 0; t < n_eval; ++t)
    for (int k = 0; k < 4; ++k) sums[k] += ui[4 * t + k];
  free(ui);
  if (U_real) *U_real = 0.5 * sums[0];
  if (U_lj) *U_lj = 0.5 * sums[1];
  if (W_real) *W_real = 0.5 * sums[2];
  if (W_lj) *W_lj = 0.5 * sums[3];
  return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Linked cells (Sec. 2.2: linked-cell reassignment and cell-wise reordering): stable
 * counting sort of ids by cell; input order is ascending id, so each cell lists its
 * particles in ascending id. */
int orc_cells(int64_t N, const uint32_t *s, const int32_t n[3], int32_t *cell_of,
              int64_t *cell_start, int64_t *sorted_ids) {
  if (N < 0 || n[0] < 1 || n[1] < 1 || n[2] < 1) return -1;
  int64_t ncell = (int64_t)n[0] * n[1] * n[2];
  for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = 0;
  for (int64_t i = 0; i < N; ++i) {
    int64_t c[3];
    for (int d = 0; d < 3; ++d) c[d] = (int64_t)(((uint64_t)s[3 * i + d] * (uint64_t)n[d]) >> 32);
    cell_of[i] = (int32_t)(c[0] + (int64_t)n[0] * (c[1] + (int64_t)n[1] * c[2]));
    cell_start[cell_of[i] + 1] += 1;
  }
  for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
  for (int64_t c = 0; c < ncell; ++c) fill[c] = cell_start[c];
  for (int64_t i = 0; i < N; ++i) sorted_ids[fill[cell_of[i]]++] = i;
  free(fill);
  return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Random batch list, Eqs. Ci_Si, RBL and F_corr. */
/* The r_s grid of the random batch list (n_d = floor(L_d / r_s) cells, at least 3 per axis,
 * 2 r_s < L_d) with the members of every cell in ascending (s_x, id) order, the canonical
 * order the draws index (the paper leaves the order inside a cell open). Returns -3 when the
 * box is too small; otherwise the three arrays are the caller's to free. */
static int rbl_grid(int64_t N, const uint32_t *s, const double box[3], double r_s,
                    int32_t n[3], int32_t **cell_of_out, int64_t **cell_start_out,
                    int64_t **sorted_ids_out) {
  for (int d = 0; d < 3; ++d) {
    n[d] = (int32_t)floor(box[d] / r_s);
    if (n[d] < 3 || !(2.0 * r_s < box[d])) return -3;
  }
  int64_t ncell = (int64_t)n[0] * n[1] * n[2];
  int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  int64_t *cell_start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
  int64_t *sorted_ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  orc_cells(N, s, n, cell_of, cell_start, sorted_ids);
  for (int64_t cc = 0; cc < ncell; ++cc)
    for (int64_t k = cell_start[cc] + 1; k < cell_start[cc + 1]; ++k) {
      const int64_t v = sorted_ids[k];
      int64_t u = k - 1;
      while (u >= cell_start[cc] &&
             (s[3 * sorted_ids[u]] > s[3 * v] ||
              (s[3 * sorted_ids[u]] == s[3 * v] && sorted_ids[u] > v))) {
        sorted_ids[u + 1] = sorted_ids[u];
        --u;
      }
      sorted_ids[u + 1] = v;
    }
  *cell_of_out = cell_of;
  *cell_start_out = cell_start;
  *sorted_ids_out = sorted_ids;
  return 0;
}

/* Row i of the random batch list before the mean-force correction (Eqs. Ci_Si, RBL): the
 * core sum, the shell in canonical order, the draws and the weighted shell sum. f receives
 * F~_i, u the weighted per-i sums of (U_real, U_lj, W_real, W_lj), *nc and *ns the set
 * sizes, partners_i (nullable, p entries) the drawn ids (-1 when unused). *shell / *cap is
 * the caller's scratch, grown as needed. */
static void rbl_row(int64_t i, const uint32_t *s, const double *q, const int32_t *type,
                    const double box[3], double alpha, double rcore2, double rs2, int p,
                    const uint32_t key[2], uint64_t step, double C, int ntypes,
                    const double *eps, const double *sig, const int32_t n[3],
                    const int32_t *cell_of, const int64_t *cell_start,
                    const int64_t *sorted_ids, int64_t **shell, int64_t *cap, double f_out[3],
                    double u_out[4], int64_t *nc_out, int64_t *ns_out, int32_t *partners_i) {
  int64_t ci = cell_of[i];
  int64_t c3[3] = {ci % n[0], (ci / n[0]) % n[1], ci / ((int64_t)n[0] * n[1])};
  double f[3] = {0.0, 0.0, 0.0}, acc[4] = {0.0, 0.0, 0.0, 0.0};
  int64_t ns = 0, nc = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t cx = (c3[0] + dx + n[0]) % n[0];
        int64_t cy = (c3[1] + dy + n[1]) % n[1];
        int64_t cz = (c3[2] + dz + n[2]) % n[2];
        int64_t cj = cx + (int64_t)n[0] * (cy + (int64_t)n[1] * cz);
        for (int64_t k = cell_start[cj]; k < cell_start[cj + 1]; ++k) {
          int64_t j = sorted_ids[k];
          if (j == i) continue;
          double d[3];
          double r2 = orc_min_image_r2(&s[3 * i], &s[3 * j], box, d);
          if (r2 <= rcore2) {
            ++nc;
            int pt = type[i] * ntypes + type[j];
            double g, a, b, c, e;
            pair_terms(r2, q[i] * q[j], alpha, C, eps[pt], sig[pt], &g, &a, &b, &c, &e);
            for (int kk = 0; kk < 3; ++kk) f[kk] += g * d[kk];
            acc[0] += a; acc[1] += b; acc[2] += c; acc[3] += e;
          } else if (r2 <= rs2) {
            if (ns == *cap) {
              *cap *= 2;
              *shell = (int64_t *)realloc(*shell, sizeof(int64_t) * (size_t)*cap);
            }
            (*shell)[ns++] = j;
          }
        }
      }
  /* shell part: all partners with weight 1 when n_s <= p, else p i.i.d. draws */
  double fs[3] = {0.0, 0.0, 0.0}, as[4] = {0.0, 0.0, 0.0, 0.0};
  double weight = 1.0;
  int64_t nuse = ns <= p ? ns : p;
  if (ns > p) weight = (double)ns / (double)p;
  for (int64_t t = 0; t < nuse; ++t) {
    int64_t j;
    if (ns <= p) {
      j = (*shell)[t];
    } else {
      uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(t / 4), (uint32_t)step, 1u};
      uint32_t w[4];
      orc_philox4x32_10(ctr, key, w);
      uint64_t idx = ((uint64_t)w[t % 4] * (uint64_t)ns) >> 32;
      j = (*shell)[idx];
    }
    if (partners_i) partners_i[t] = (int32_t)j;
    double d[3];
    double r2 = orc_min_image_r2(&s[3 * i], &s[3 * j], box, d);
    int pt = type[i] * ntypes + type[j];
    double g, a, b, c, e;
    pair_terms(r2, q[i] * q[j], alpha, C, eps[pt], sig[pt], &g, &a, &b, &c, &e);
    for (int kk = 0; kk < 3; ++kk) fs[kk] += g * d[kk];
    as[0] += a; as[1] += b; as[2] += c; as[3] += e;
  }
  if (partners_i)
    for (int64_t t = nuse; t < p; ++t) partners_i[t] = -1;
  for (int kk = 0; kk < 3; ++kk) f_out[kk] = f[kk] + weight * fs[kk];
  for (int kk = 0; kk < 4; ++kk) u_out[kk] = acc[kk] + weight * as[kk];
  *nc_out = nc;
  *ns_out = ns;
}

int orc_rbl(int64_t N, const uint32_t *s, const double *q, const int32_t *type,
            const double box[3], double alpha, double r_core, double r_s, int p,
            uint64_t seed, uint64_t step, uint32_t replica, double C, int ntypes,
            const double *eps, const double *sig, double *F, double *U_real,
            double *U_lj, double *W_real, double *W_lj, int32_t *n_core,
            int32_t *n_shell, int32_t *partners) {
  if (N <= 0 || p < 1 || !(r_core >= 0) || !(r_s > r_core) || ntypes < 1) return -1;
  int32_t n[3], *cell_of;
  int64_t *cell_start, *sorted_ids;
  int grc = rbl_grid(N, s, box, r_s, n, &cell_of, &cell_start, &sorted_ids);
  if (grc) return grc;
  double rcore2 = r_core * r_core, rs2 = r_s * r_s;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ replica};
  double *Ft = (double *)malloc(sizeof(double) * 3 * (size_t)N);
  double *ui = (double *)calloc((size_t)N * 4, sizeof(double));
  int bad = 0;
#pragma omp parallel
  {
    int64_t cap = 1024;
    int64_t *shell = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
      int64_t nc, ns;
      rbl_row(i, s, q, type, box, alpha, rcore2, rs2, p, key, step, C, ntypes, eps, sig, n,
              cell_of, cell_start, sorted_ids, &shell, &cap, &Ft[3 * i], &ui[4 * i], &nc, &ns,
              partners ? &partners[(int64_t)p * i] : NULL);
      if (n_core) n_core[i] = (int32_t)nc;
      if (n_shell) n_shell[i] = (int32_t)ns;
      if (nc > 2147483647 || ns > 2147483647) bad = 1;
    }
    free(shell);
  }
  /* momentum-conserving correction, Eq. F_corr */
  double mean[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < 3; ++k) mean[k] += Ft[3 * i + k];
  for (int k = 0; k < 3; ++k) mean[k] /= (double)N;
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < 3; ++k) F[3 * i + k] = Ft[3 * i + k] - mean[k];
  double sums[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < 4; ++k) sums[k] += ui[4 * i + k];
  if (U_real) *U_real = 0.5 * sums[0];
  if (U_lj) *U_lj = 0.5 * sums[1];
  if (W_real) *W_real = 0.5 * sums[2];
  if (W_lj) *W_lj = 0.5 * sums[3];
  free(cell_of); free(cell_start); free(sorted_ids); free(Ft); free(ui);
  return bad ? -4 : 0;
}

/* Rows i_list[0..n_list) of the random batch list before the mean-force correction, with
 * the grid, enumeration and draws of orc_rbl: Ft (n_list x 3) receives F~_i, u (nullable,
 * n_list x 4) the weighted per-i sums of (U_real, U_lj, W_real, W_lj), n_core / n_shell
 * (nullable, n_list) the set sizes and partners (nullable, n_list x p) the drawn ids. The
 * correction -(1/N) sum_j F~_j of Eq. F_corr needs every row, so a sample of rows sees it
 * as one offset common to all of them. */
int orc_rbl_rows(int64_t N, const uint32_t *s, const double *q, const int32_t *type,
                 const double box[3], double alpha, double r_core, double r_s, int p,
                 uint64_t seed, uint64_t step, uint32_t replica, double C, int ntypes,
                 const double *eps, const double *sig, const int64_t *i_list, int64_t n_list,
                 double *Ft, double *u, int32_t *n_core, int32_t *n_shell,
                 int32_t *partners) {
  if (N <= 0 || p < 1 || !(r_core >= 0) || !(r_s > r_core) || ntypes < 1 || n_list < 0)
    return -1;
  for (int64_t t = 0; t < n_list; ++t)
    if (i_list[t] < 0 || i_list[t] >= N) return -1;
  int32_t n[3], *cell_of;
  int64_t *cell_start, *sorted_ids;
  int grc = rbl_grid(N, s, box, r_s, n, &cell_of, &cell_start, &sorted_ids);
  if (grc) return grc;
  double rcore2 = r_core * r_core, rs2 = r_s * r_s;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ replica};
  int bad = 0;
#pragma omp parallel
  {
    int64_t cap = 1024;
    int64_t *shell = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < n_list; ++t) {
      int64_t nc, ns;
      double ut[4];
      rbl_row(i_list[t], s, q, type, box, alpha, rcore2, rs2, p, key, step, C, ntypes, eps,
              sig, n, cell_of, cell_start, sorted_ids, &shell, &cap, &Ft[3 * t], ut, &nc, &ns,
              partners ? &partners[(int64_t)p * t] : NULL);
      if (u)
        for (int kk = 0; kk < 4; ++kk) u[4 * t + kk] = ut[kk];
      if (n_core) n_core[t] = (int32_t)nc;
      if (n_shell) n_shell[t] = (int32_t)ns;
      if (nc > 2147483647 || ns > 2147483647) bad = 1;
    }
    free(shell);
  }
  free(cell_of); free(cell_start); free(sorted_ids);
  return bad ? -4 : 0;
}

/* ---------------------------------------------------------------------------------- */
/* Brute-force lattice sum of Eq. Coul_potential over whole image cells n whose shift
 * n o L lies in the sphere of radius R L_x, then converted to tin-foil boundary
 * conditions (the spherical sum converges to the Ewald sum plus the surface term). */
int orc_brute_coulomb(int64_t N, const uint32_t *s, const double *q, const double box[3],
                      double C, int R, double *F, double *U) {
  if (N < 0 || R < 0) return -1;
  double V = box[0] * box[1] * box[2];
  double Mdip[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < N; ++i) {
    double r[3];
    position(&s[3 * i], box, r);
    for (int d = 0; d < 3; ++d) Mdip[d] += q[i] * r[d];
  }
  double *ui = (double *)calloc((size_t)N, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < N; ++i) {
    double ri[3], f[3] = {0.0, 0.0, 0.0}, u = 0.0;
    position(&s[3 * i], box, ri);
    double Rl = (double)R * box[0]; /* radius of the sphere of image cells */
    int nb[3];
    for (int k = 0; k < 3; ++k) nb[k] = (int)ceil(Rl / box[k]);
    for (int nz = -nb[2]; nz <= nb[2]; ++nz)
      for (int ny = -nb[1]; ny <= nb[1]; ++ny)
        for (int nx = -nb[0]; nx <= nb[0]; ++nx) {
          double ex = nx * box[0], ey = ny * box[1], ez = nz * box[2];
          if (ex * ex + ey * ey + ez * ez > Rl * Rl) continue;
          for (int64_t j = 0; j < N; ++j) {
            if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
            double rj[3], d[3];
            position(&s[3 * j], box, rj);
            d[0] = ri[0] - rj[0] + nx * box[0];
            d[1] = ri[1] - rj[1] + ny * box[1];
            d[2] = ri[2] - rj[2] + nz * box[2];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            u += q[j] / r;
            for (int k = 0; k < 3; ++k) f[k] += q[j] * d[k] / (r2 * r);
          }
        }
    for (int k = 0; k < 3; ++k)
      F[3 * i + k] = C * q[i] * f[k] + 4.0 * M_PI * C * q[i] * Mdip[k] / (3.0 * V);
    ui[i] = q[i] * u;
  }
  double u = 0.0;
  for (int64_t i = 0; i < N; ++i) u += ui[i];
  free(ui);
  double M2 = Mdip[0] * Mdip[0] + Mdip[1] * Mdip[1] + Mdip[2] * Mdip[2];
  *U = 0.5 * C * u - 2.0 * M_PI * C * M2 / (3.0 * V);
  return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Velocity Verlet (the "prescribed time integrator" of Sec. 2.1) on the fixed-point grid. */
int orc_vv_drift(int64_t N, uint32_t *s, double *v, const double *F, const double *mass,
                 const double box[3], double dt, double kappa) {
  if (N < 0) return -1;
  for (int64_t i = 0; i < N; ++i) {
    for (int d = 0; d < 3; ++d) {
      v[3 * i + d] += F[3 * i + d] / mass[i] * (0.5 * dt) * kappa;
      double ds = v[3 * i + d] * dt * TWO32 / box[d];
      long long step = llrint(ds);
      s[3 * i + d] = (uint32_t)(s[3 * i + d] + (uint32_t)(int64_t)step);
    }
  }
  return 0;
}

int orc_vv_kick(int64_t N, double *v, const double *F, const double *mass, double dt,
                double kappa) {
  if (N < 0) return -1;
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) v[3 * i + d] += F[3 * i + d] / mass[i] * (0.5 * dt) * kappa;
  return 0;
}

/* Nose-Hoover thermostat half step (chain of one), Trotter-split around the Verlet step. */
int orc_nh_half(int64_t N, double *v, const double *mass, double kappa, double Nf, double kT,
                double Q, double dt, double xi_eta[2]) {
  if (N < 0 || !(Q > 0)) return -1;
  double K2 = 0.0; /* 2K = sum m v^2 / kappa */
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) K2 += mass[i] * v[3 * i + d] * v[3 * i + d] / kappa;
  double xi = xi_eta[0];
  xi += 0.25 * dt * (K2 - Nf * kT) / Q;
  double s = exp(-xi * 0.5 * dt);
  for (int64_t i = 0; i < 3 * N; ++i) v[i] *= s;
  K2 *= s * s;
  xi_eta[1] += xi * 0.5 * dt;
  xi += 0.25 * dt * (K2 - Nf * kT) / Q;
  xi_eta[0] = xi;
  return 0;
}
