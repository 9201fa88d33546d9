/*
 * rbe_oracle.h -- plain FP64 CPU oracle for the improved random batch Ewald (RBE)
 * nonbonded force path of RBMD 2.0 (Gao et al., arXiv 2609.02694).
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA path. Only the test
 * suite, __graft_entry__.smoke() and the cpu_baseline / reference leg of bench.py load
 * it. The product library never links, calls or reads anything from here, and this
 * code shares no source, header, table or constant generator with it.
 *
 * Conventions shared by every entry point:
 *   - N particles; positions are given on the 2^-32 fractional grid as uint32 triples
 *     s[3*i + d], so r_d = s_d * L_d / 2^32 exactly (the reading of the paper's
 *     positions adopted by this build; see the design notes).
 *   - box[3] = (L_x, L_y, L_z), orthorhombic, periodic in all three directions (Sec. 2.1).
 *   - q[i] charges in units of e, C the Coulomb constant (energy*length/e^2).
 *   - LJ parameters per type pair: eps[ti*ntypes + tj], sig[ti*ntypes + tj] (Eq. LJ).
 *   - alpha is the paper's Ewald parameter, of units length^-2 (Eqs. Ewald, U_Coul_Fourier).
 *   - All arithmetic is IEEE FP64, compiled without FMA contraction, summed in a fixed
 *     order (ascending particle id, ascending mode index).
 *   - Functions return 0 on success and a negative value on invalid input.
 *
 * Parity status of each function is stated beside it: "pinned by ..." names the
 * independent checks in tests/test_oracle_*.py.
 */
#ifndef RBE_ORACLE_H
#define RBE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).
 * Pinned by the published known-answer vectors. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Half-width M of the per-dimension mode table: the smallest integer with
 * exp(-(2 pi M / L)^2 / (4 alpha)) below 2^-53. */
int orc_kdim_M(double L, double alpha);

/* Cumulative thresholds of the 1-D discrete Gaussian exp(-k^2/(4 alpha)), k = 2 pi m / L,
 * m = -M..M (the factor of the sampling density of Sec. 2.1, Eq. F_long_RBE, along one
 * axis). T[i] = floor(CDF(m_i) / Z * 2^32) with the last entry 2^32; *Z = sum of weights.
 * Pinned by the Poisson-summation closed form of Z and a chi-square test of the draws. */
int orc_kdim_table(double L, double alpha, int M, uint64_t *T, double *Z);

/* Importance sampling of P modes from P(k) ~ exp(-k^2/4 alpha), k != 0 (Eq. F_long_RBE):
 * mode l draws Philox(counter = (l, attempt, step_lo32, 0), key = (seed_lo32,
 * seed_hi32 ^ replica)); word d picks m_d by inverse CDF on the table of axis d; the draw is
 * rejected and redrawn with attempt+1 when m = 0. m[3*l + d] receives the integers,
 * *S = Z_x Z_y Z_z - 1 the normaliser. Returns -2 if 64 attempts all gave m = 0. */
int orc_sample_k(uint64_t seed, uint64_t step, uint32_t replica, const double box[3],
                 double alpha, int P, int32_t *m, double *S);

/* Structure factor rho(k_l) = sum_j q_j exp(i k_l . r_j) (Eq. U_Coul_Fourier);
 * rho[2l] = Re, rho[2l+1] = Im. */
int orc_rho(int64_t N, const uint32_t *s, const double *q, const double box[3], int P,
            const int32_t *m, double *rho);

/* RBE k-space force estimator on a given mode set (Eq. F_long_RBE with the leading minus
 * of Eq. F_i, the reading adopted for the sign), the matching energy estimator
 * (S/P) sum_l 2 pi C |rho_l|^2 / (V k_l^2) and its scalar virial
 * sum_l E_l (1 - k_l^2 / (2 alpha)). F is overwritten (N x 3).
 * Pinned by zero net force, finite differences of the energy, and unbiasedness against
 * the full Ewald sum over 10^4 seeds. */
int orc_rbe_kspace(int64_t N, const uint32_t *s, const double *q, const double box[3],
                   double alpha, double C, int P, const int32_t *m, double S,
                   double *F, double *U, double *W);

/* Full Ewald k-space sum over all m != 0 with |m_d| <= M_d (Eqs. U_Coul_Fourier, F_i).
 * Pinned by the NaCl Madelung constant, brute-force image sums and alpha-invariance. */
int orc_ewald_kspace(int64_t N, const uint32_t *s, const double *q, const double box[3],
                     double alpha, double C, double *F, double *U, double *W);
/* Full Ewald truncated at weight tol: modes k != 0 with exp(-k^2 / 4 alpha) >= tol only. */
int orc_ewald_kspace_tol(int64_t N, const uint32_t *s, const double *q, const double box[3],
                         double alpha, double C, double tol, double *F, double *U, double *W);

/* Self energy C sqrt(alpha/pi) sum q^2 (Eq. U_self). */
double orc_self_energy(int64_t N, const double *q, double alpha, double C);

/* Squared minimum-image distance used for every cutoff decision:
 * dx_d = (double)(int32)(s_i,d - s_j,d) * (L_d / 2^32), r2 = dx^2 + dy^2 + dz^2,
 * left to right, no FMA. */
double orc_min_image_r2(const uint32_t *si, const uint32_t *sj, const double box[3],
                        double d[3]);

/* Real-space part (Eqs. F_i, G_short, LJ): for every particle i the sum over all j != i
 * with r_ij <= r_c (minimum image) of (C q_i q_j G(r) + G_LJ(r)) (r_i - r_j).
 * Energies are halves of the per-i sums: U_real = 1/2 sum C q_i q_j erfc(sqrt(alpha) r)/r,
 * U_lj = 1/2 sum 4 eps((sig/r)^12 - (sig/r)^6) (plain truncation), W = 1/2 sum F_ij . r_ij.
 * If i_list is non-NULL only the n_list particles it names are evaluated (O(N) each) and F
 * rows are written for those only; energies then cover those particles' halves.
 * nbr_count (nullable) receives the number of j within the cutoff per evaluated i.
 * Pinned by finite differences, the LJ zero-force distance, the alpha -> 0 limit and the
 * brute-force image sum. */
int orc_real_space(int64_t N, const uint32_t *s, const double *q, const int32_t *type,
                   const double box[3], double alpha, double rc, double C, int ntypes,
                   const double *eps, const double *sig, const int64_t *i_list,
                   int64_t n_list, double *F, double *U_real, double *U_lj,
                   double *W_real, double *W_lj, int32_t *nbr_count);

/* Linked cells: n[d] cells per axis, cell of i = c_x + n_x (c_y + n_y c_z) with
 * c_d = floor(s_d n_d / 2^32); particles ordered by (cell, id). cell_start has
 * n_x n_y n_z + 1 entries; sorted_ids[k] is the id at sorted position k. */
int orc_cells(int64_t N, const uint32_t *s, const int32_t n[3], int32_t *cell_of,
              int64_t *cell_start, int64_t *sorted_ids);

/* Random batch list (Eqs. Ci_Si, RBL, F_corr) on the r_s grid (n_d = floor(L_d / r_s)
 * cells, at least 3 per axis). For particle i the candidates are enumerated over the 27
 * neighbour cells in (dz, dy, dx) order, each from -1 to 1, and inside a cell in
 * ascending (s_x, id) order; j != i with r <= r_core is core, r_core < r <= r_s is shell. With
 * n_s = #shell: if n_s <= p all shell partners enter with weight 1; otherwise p draws
 * idx = floor(w * n_s / 2^32), w = word (t mod 4) of Philox(counter = (id_i, t / 4,
 * step_lo32, 1), key = (seed_lo32, seed_hi32 ^ replica)), t = 0..p-1, each entering with
 * weight n_s / p. F receives the corrected force F~_i - (1/N) sum_j F~_j (N x 3);
 * energies and virial are halves of the weighted per-i sums. n_core / n_shell (nullable)
 * receive the set sizes; partners (nullable, N x p) the drawn ids (-1 when unused).
 * Pinned by the exact limits r_core = r_s and p >= n_s, zero net force and
 * unbiasedness over seeds. */
int orc_rbl(int64_t N, const uint32_t *s, const double *q, const int32_t *type,
            const double box[3], double alpha, double r_core, double r_s, int p,
            uint64_t seed, uint64_t step, uint32_t replica, double C, int ntypes,
            const double *eps, const double *sig, double *F, double *U_real,
            double *U_lj, double *W_real, double *W_lj, int32_t *n_core,
            int32_t *n_shell, int32_t *partners);

/* Rows i_list[0..n_list) (ids in [0, N)) of the random batch list before the mean-force
 * correction: the grid, enumeration, draws and weights of orc_rbl for those rows only.
 * Ft (n_list x 3) receives F~_i, u (nullable, n_list x 4) the weighted per-i sums of
 * (U_real, U_lj, W_real, W_lj), n_core / n_shell (nullable) the set sizes and partners
 * (nullable, n_list x p) the drawn ids (-1 when unused). The correction -(1/N) sum_j F~_j
 * needs every row: for a sample it is one offset common to all rows. Returns -1 on an
 * invalid argument or id, -3 when the box holds fewer than 3 cells of r_s per axis. */
int orc_rbl_rows(int64_t N, const uint32_t *s, const double *q, const int32_t *type,
                 const double box[3], double alpha, double r_core, double r_s, int p,
                 uint64_t seed, uint64_t step, uint32_t replica, double C, int ntypes,
                 const double *eps, const double *sig, const int64_t *i_list, int64_t n_list,
                 double *Ft, double *u, int32_t *n_core, int32_t *n_shell,
                 int32_t *partners);

/* Brute-force Coulomb lattice sum of Eq. Coul_potential over whole image cells with
 * |n o L| <= R L_x (spherical order), converted to the tin-foil convention of the Ewald sum by
 * subtracting 2 pi |M|^2 / (3V) from the energy and adding 4 pi q_i M / (3V) to the
 * force (M = sum_i q_i r_i). Used only as a pin. */
int orc_brute_coulomb(int64_t N, const uint32_t *s, const double *q, const double box[3],
                      double C, int R, double *F, double *U);

/* One velocity-Verlet step on the fixed-point grid with forces supplied by the caller:
 * v += (F/m)(dt/2) kappa; s += round(v dt 2^32 / L) (mod 2^32). The second half-kick is
 * a separate call (orc_vv_kick) once the new forces are known. */
int orc_vv_drift(int64_t N, uint32_t *s, double *v, const double *F, const double *mass,
                 const double box[3], double dt, double kappa);
int orc_vv_kick(int64_t N, double *v, const double *F, const double *mass, double dt,
                double kappa);

/* Nose-Hoover half step (chain of one thermostat, Trotter splitting of the Liouville
 * operator): xi += dt/4 (2K - Nf kT)/Q; v *= exp(-xi dt/2); eta += xi dt/2;
 * xi += dt/4 (2K' - Nf kT)/Q, with K = 1/2 sum m v^2 / kappa before and K' after the
 * scaling. xi_eta[2] = {xi, eta} is updated in place. Applied before the first half-kick
 * and after the second of every velocity-Verlet step. */
int orc_nh_half(int64_t N, double *v, const double *mass, double kappa, double Nf, double kT,
                double Q, double dt, double xi_eta[2]);

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int orc_num_threads(void);

/* Set the number of OpenMP threads for later calls (n >= 1; no effect without OpenMP),
 * for timing the oracle on one core and on all of them. Results do not depend on it. */
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
