/*
 * rbe.h -- C ABI of the GB300-native improved random batch Ewald (RBE) force path.
 *
 * The library evaluates the nonbonded force of RBMD 2.0 (arXiv 2609.02694, Sec. 2.1) for
 * point charges with Lennard-Jones interactions in an orthorhombic periodic box:
 *   F_i = F_i^N + F_i^F                                   (Eq. F_i)
 * where F^N is the erfc-screened Coulomb + LJ pair force inside the cutoff (Eqs. F_i,
 * G_short, LJ), evaluated over linked cells or by the random batch list (Eqs. Ci_Si, RBL,
 * F_corr), and F^F is the importance-sampled k-space estimator (Eq. F_long_RBE) on P modes
 * drawn from P(k) ~ exp(-k^2 / 4 alpha), k != 0.
 *
 * Conventions
 *  - Units are the caller's. The Coulomb constant, the force-to-acceleration factor and
 *    the time step are parameters. Real units (Angstrom, fs, amu, kcal/mol, e) use
 *    coulomb_C = 332.06371 and kappa = 4.184e-4.
 *  - alpha is the paper's Ewald parameter, in length^-2 (Eq. Ewald: erfc(sqrt(alpha) r)).
 *  - Positions are stored on the 2^-32 fractional grid: s_d = round(r_d / L_d * 2^32) mod
 *    2^32. Positions that are already on that grid are kept exactly.
 *  - Arrays of N x 3 values are row-major per particle (x, y, z) and indexed by the
 *    caller's particle id 0..N-1. The library reorders particles internally by cell and
 *    translates back on every output.
 *  - Every call returns RBE_OK (0) or a negative RBE_ERR_* code. rbe_error_string() gives
 *    a message. A failed call leaves the handle usable unless it returns RBE_ERR_CUDA.
 *  - Calls are asynchronous on the stream given to rbe_init, except those that return
 *    host data. Those synchronise that stream before they return.
 *  - The library owns every device buffer it allocates and frees them in rbe_destroy.
 *    Caller buffers are never retained after a call returns.
 */
#ifndef RBE_H
#define RBE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbe_ctx *rbe_handle;

enum {
  RBE_OK = 0,
  RBE_ERR_INVALID = -1,     /* a NULL handle or pointer, or a value out of range */
  RBE_ERR_NONNEUTRAL = -2,  /* |sum q| > 1e-9 * max(1, sum |q|) (charge neutrality, Sec. 2.1) */
  RBE_ERR_CUTOFF = -3,      /* r_c >= L/2 on some axis (minimum image not unique) */
  RBE_ERR_CELLS = -4,       /* fewer cells per axis than the stencil needs */
  RBE_ERR_OOM = -5,         /* device allocation failed */
  RBE_ERR_CUDA = -6,        /* a CUDA runtime error; the handle should be destroyed */
  RBE_ERR_SAMPLER = -7,     /* 64 redraws of a mode all gave k = 0 (device flag) */
  RBE_ERR_NONFINITE = -8,   /* a non-finite velocity or position update (device flag) */
  RBE_ERR_STATE = -9,       /* call not valid in this state (e.g. no forces computed yet) */
  RBE_ERR_CAPACITY = -10    /* an RBL stencil (27 cells) held more than 6144 candidates, or a
                               Verlet list outgrew its capacity (device flag) */
};

enum {
  RBE_FP32_COMP = 0, /* FP32 pair and phase math; compensated FP32 partials, FP64 combine */
  RBE_FP32 = 1,      /* plain FP32 everywhere, partials combined in FP32 */
  RBE_FP64 = 2       /* FP64 pair, phase and trig math, FP64 accumulation */
};

/* Energies written by rbe_forces (all in the caller's energy unit). */
enum {
  RBE_E_REAL = 0,  /* U^N Coulomb: 1/2 sum C q_i q_j erfc(sqrt(alpha) r)/r over r <= r_c */
  RBE_E_LJ = 1,    /* U_LJ of Eq. LJ, plainly truncated at r_c */
  RBE_E_KSPACE = 2,/* RBE estimator of Eq. U_Coul_Fourier: (S/P) sum_l 2 pi C |rho_l|^2/(V k_l^2) */
  RBE_E_SELF = 3,  /* Eq. U_self: C sqrt(alpha/pi) sum q^2 */
  RBE_E_TOTAL = 4, /* REAL + LJ + KSPACE - SELF */
  RBE_E_KINETIC = 5,/* 1/2 sum m v^2 / kappa at the current velocities */
  RBE_N_ENERGY = 6
};

/* Scalar virials W = sum r . F (W_k from the homogeneity of U^F: sum_l E_l (1 - k_l^2/2 alpha)). */
enum { RBE_W_REAL = 0, RBE_W_LJ = 1, RBE_W_KSPACE = 2, RBE_W_TOTAL = 3, RBE_N_VIRIAL = 4 };

typedef struct {
  double alpha;        /* Ewald splitting parameter, length^-2 (Eq. Ewald) */
  double r_c;          /* real-space cutoff: the paper's r_s in Eq. Ci_Si (and r_c of Eq. F_i) */
  double r_core;       /* RBL core radius, the paper's r_c of Eq. Ci_Si; 0 selects the plain
                          cell-list real space */
  int32_t p_rbl;       /* RBL shell batch size p (Eq. RBL); used when r_core > 0 */
  int32_t P;           /* number of sampled Fourier modes (Eq. F_long_RBE), >= 1 */
  uint64_t seed;       /* Philox key for the mode and RBL draws */
  uint32_t replica;    /* xored into the upper key word: independent streams per replica */
  int32_t precision;   /* RBE_FP32_COMP, RBE_FP32 or RBE_FP64 */
  double coulomb_C;    /* Coulomb constant C (energy x length / charge^2) */
  double dt;           /* time step of rbe_step */
  double kappa;        /* force / mass -> acceleration factor of rbe_step */
  int32_t n_types;     /* number of LJ types, 1..16 */
  const double *lj_eps;   /* n_types x n_types, symmetric (Eq. LJ epsilon_ij) */
  const double *lj_sigma; /* n_types x n_types, symmetric (Eq. LJ sigma_ij) */
  int32_t cell_sub;    /* real-space cells per cutoff length (1, 2 or 3); 0 = library default */
} rbe_params;

/* Create a handle for N particles in box[3] (orthorhombic side lengths).
 *  pos   N x 3 positions (host), wrapped into the box and quantised to the 2^-32 grid
 *  q     N charges (host); the system must be neutral
 *  type  N LJ type indices in [0, n_types) (host), or NULL for all type 0
 *  mass  N masses (host), or NULL when rbe_step is not used (mass 1)
 *  vel   N x 3 velocities (host), or NULL for zero
 *  cuda_stream  a cudaStream_t the library launches on (NULL = legacy default stream)
 * Allocates all device memory for the system; later calls allocate nothing, except
 * rbe_set_neighbor_list (the list buffers) and rbe_measure_peak (64 bytes of scratch). */
int rbe_init(rbe_handle *h, const rbe_params *p, int64_t N, const double box[3],
             const double *pos, const double *q, const int32_t *type, const double *mass,
             const double *vel, void *cuda_stream);

/* Draw the P modes of step `step` (Eq. F_long_RBE; the sampling density of Sec. 2.1) on the
 * device and, if m_out (host, P x 3 int32) is non-NULL, copy them back; *S_out (nullable)
 * receives the normaliser S = sum_{k != 0} exp(-k^2 / 4 alpha). Mode l is a pure function
 * of (seed, replica, step, l) (Philox4x32-10 counter (l, attempt, step, 0)), which plays
 * the role of the paper's broadcast seed (Sec. 2.3.1). */
int rbe_sample_k(rbe_handle h, uint64_t step, int32_t *m_out, double *S_out);

/* Replace the positions (N x 3, in id order) from host (on_device = 0) or device memory. */
int rbe_set_positions(rbe_handle h, const double *pos, int on_device);

/* One nonbonded force evaluation for step `step`: F_i = F_i^N (real space, Eqs. F_i,
 * G_short and LJ over r <= r_c; or the random batch list, Eqs. Ci_Si and RBL, with the
 * mean-force correction of Eq. F_corr when r_core > 0) + F_i^{F,*} (the random batch Ewald
 * k-space force, Eq. F_long_RBE, on this step's modes), with the energies of Eqs.
 * U_Coul_Fourier and U_self. Stages: bin + sort (Sec. 2.2) -> sample P modes -> structure
 * factor -> real space -> k-space gather -> totals.
 *  F_out     N x 3 float forces in id order (nullable), in host (F_on_device = 0) or
 *            device memory
 *  energies  RBE_N_ENERGY doubles (nullable, host)
 *  virial    RBE_N_VIRIAL doubles (nullable, host)
 * The call synchronises when any host output is requested. With profiling off, the stages
 * run as a CUDA graph captured at the first call on each of the two buffer parities (an
 * internal stream is captured; make those first calls outside any stream capture of the
 * caller's own) and replayed afterwards; the step number is written to the device before
 * each replay. The graphs are captured again after a change of tuning, profiling, neighbour
 * list or thermostat, or a checkpoint load. */
int rbe_forces(rbe_handle h, uint64_t step, float *F_out, int F_on_device, double *energies,
               double *virial);

/* Same as rbe_forces, with FP64 forces written to host memory (for parity checks); it also
 * records the neighbour counts and RBL draws that rbe_get_neighbor_counts and
 * rbe_get_rbl_partners return. It always launches its stages one by one (no graph). */
int rbe_forces_f64(rbe_handle h, uint64_t step, double *F_out, double *energies,
                   double *virial);

/* Advance nsteps velocity-Verlet steps (the time integrator of Sec. 2.1: kick-drift,
 * forces as rbe_forces computes them, kick) from the current step counter, replaying one
 * captured CUDA graph per step; asynchronous. The first call computes the initial forces
 * if none exist and captures the graph. */
int rbe_step(rbe_handle h, int nsteps);

/* Energies and virials of the last force evaluation or Verlet step (host, nullable each;
 * RBE_N_ENERGY and RBE_N_VIRIAL doubles): real-space Coulomb and LJ sums, the k-space
 * estimate of Eq. U_Coul_Fourier on the sampled modes, the self energy of Eq. U_self and
 * the kinetic energy. Synchronises the stream. */
int rbe_get_energies(rbe_handle h, double *energies, double *virial);

/* Nose-Hoover NVT thermostat for rbe_step (the NVT runs of Sec. 3; a chain of one
 * thermostat, Trotter-split
 * around each velocity-Verlet step: half step before the first half-kick and after the
 * second). Q = N_f kB T tau^2 with N_f = 3N - 3. tau <= 0 switches it off (NVE, the
 * default). kB is in the caller's energy unit per kelvin (0.0019872067 for kcal/mol).
 * The friction xi and the integral eta start at 0; calling again resets them. */
int rbe_set_thermostat(rbe_handle h, double T_target, double tau, double kB);

/* Thermostat state after the last step: out[0] = xi, out[1] = eta,
 * out[2] = Q xi^2 / 2 + N_f kB T eta (add it to U + K for the conserved quantity). */
int rbe_get_thermostat(rbe_handle h, double out[3]);

/* Current step counter (number of completed rbe_step steps). */
int rbe_get_step(rbe_handle h, uint64_t *step);

/* Copy the state back in id order (each nullable): positions (exact dequantisation of the
 * 2^-32 grid, wrapped into [0, L)), velocities, and the raw fractional coordinates. */
int rbe_get_state(rbe_handle h, double *pos, double *vel, uint32_t *s_frac);

/* Copy the linked cells (Sec. 2.2) of the last force evaluation: n_cells[3] cells per axis,
 * cell_start (n_x n_y n_z + 1 entries) and sorted_ids (N ids in cell order, inside a cell
 * by (s_x, id)). Either array may be NULL (query n_cells first to size cell_start). */
int rbe_get_cells(rbe_handle h, int32_t n_cells[3], int64_t *cell_start, int64_t *sorted_ids);

/* Copy the structure factor rho(k) = sum_j q_j exp(i k . r_j) (Eq. U_Coul_Fourier) of the
 * last evaluation, rho (P x 2: Re, Im, FP64, host), and the modes (P x 3 int32, host);
 * either pointer may be NULL. */
int rbe_get_rho(rbe_handle h, double *rho, int32_t *m_out);

/* Per-particle neighbour counts of the last rbe_forces_f64 evaluation (id order, nullable;
 * rbe_forces and rbe_step do not count):
 * plain cell list: n_core = #{j != i: r_ij <= r_c}, n_shell = 0;
 * RBL: n_core = #C_i, n_shell = #S_i (Eq. Ci_Si). Cutoff decisions are exact: the FP64
 * comparison of dx^2 + dy^2 + dz^2 with r^2, dx_d = (int32)(s_i - s_j) * (L_d / 2^32). */
int rbe_get_neighbor_counts(rbe_handle h, int32_t *n_core, int32_t *n_shell);

/* RBL draws of the last rbe_forces_f64 evaluation (Eq. RBL: p i.i.d. members of S_i, in S_i's
 * canonical order; N x p_rbl ids in id order, host; -1 where unused). */
int rbe_get_rbl_partners(rbe_handle h, int32_t *partners);

/* Phases timed by the profiler (CUDA events recorded on the library's stream). */
enum {
  RBE_PH_KICK_DRIFT = 0, /* first half-kick + drift (rbe_step only) */
  RBE_PH_BIN = 1,        /* list displacement check, linked-cell binning and reordering */
  RBE_PH_SAMPLE = 2,     /* Philox mode sampler */
  RBE_PH_SF = 3,         /* structure factor + FP64 combine */
  RBE_PH_LIST = 4,       /* neighbour structures: the Verlet-list build (zero on steps without
                            one), or the cluster-pair kernel's per-step cluster tables */
  RBE_PH_PAIR = 5,       /* main real-space kernel (cell list or Verlet list LJ[+Coulomb], or RBL) */
  RBE_PH_PAIR2 = 6,      /* charged-subset Coulomb pass, or the RBL mean-force correction */
  RBE_PH_GATHER = 7,     /* k-space force gather */
  RBE_PH_TAIL = 8,       /* second half-kick, kinetic energy and totals (with the cluster
                            kernel, first its fixed-point finish) */
  RBE_N_PHASE = 9
};

/* Turn per-phase event timing on or off (off by default). Toggling it discards the
 * captured step graph, which is captured again on the next rbe_step. With timing on, a step
 * runs its phases one after another; with it off, the captured step of the cluster-pair
 * kernel runs the k-space chain and the charged subset's Coulomb pass as a second graph
 * branch beside the pair pass (the same forces and energies bit for bit). */
int rbe_set_profiling(rbe_handle h, int enable);

/* Per-phase device times (ms, RBE_N_PHASE doubles) of the most recent force evaluation
 * or Verlet step, and the number of kernels one Verlet step launches. Synchronises. */
int rbe_get_profile(rbe_handle h, double *phase_ms, int64_t *kernels_per_step);

/* Tunables of the launch shapes (none changes results beyond FP32 rounding order; the
 * defaults: pair_test16 1, pair_cluster 1 except in the FP64 form, sf_tile by the
 * particle count, RBL ones automatic):
 *  RBE_TUNE_PAIR_TEST16  1: packed half-precision candidate pre-test in the cell-list pair
 *                        kernel (exact decision still at evaluation), 0: FP32 pre-test
 *  RBE_TUNE_SF_TILE      particles per block tile of the structure factor (32..1024, x32;
 *                        at most as many tiles as the tile chosen at rbe_init allows)
 *  RBE_TUNE_RBL_EAGER    random batch list only. 1: the classifying pass evaluates every shell
 *                        pair too, and a particle with #S_i <= p keeps that sum (bit-identical
 *                        to the draw pass); 0: shell pairs only in the draw pass. The default
 *                        is 1 when the mean shell size N/V * 4/3 pi (r_s^3 - r_core^3) <= p.
 *  RBE_TUNE_RBL_SPAN     random batch list only: cells in x that one warp's particle group may
 *                        span (1..14; 0 = automatic, floor(32 / particles per cell), at least 1,
 *                        at most n_x - 2). Results are bit-identical for every span.
 *  RBE_TUNE_PAIR_CLUSTER 1 (default): the cell-list pair pass over all particles runs over
 *                        clusters of 8 particles and evaluates each pair once (Newton's third
 *                        law), summing forces in 64-bit fixed point (results independent of the
 *                        order of the sums), where the box allows it (a cell width plus 2 r_c
 *                        below L in y and z); 0: the per-particle kernel (each pair from both
 *                        sides). Neighbour sets are the same exact ones either way. */
enum { RBE_TUNE_PAIR_TEST16 = 0, RBE_TUNE_SF_TILE = 1, RBE_TUNE_RBL_EAGER = 2,
       RBE_TUNE_RBL_SPAN = 3, RBE_TUNE_PAIR_CLUSTER = 4, RBE_N_TUNE = 5 };
int rbe_set_tuning(rbe_handle h, int key, int value);
int rbe_get_tuning(rbe_handle h, int key, int *value);

/* Autotuner: times each candidate setting of the tunables above on the handle's own system
 * (force evaluations, CUDA events, `reps` repetitions each) and keeps the fastest.
 * Discards the captured step graph. Writes the chosen values, indexed by RBE_TUNE_*, to
 * chosen[RBE_N_TUNE] (nullable). */
int rbe_autotune(rbe_handle h, int reps, int *chosen);

/* Verlet neighbour list with skin (the short-range traversal that Sec. 3.1 pairs with RBE),
 * an alternative to the per-step cell traversal of the cell-list real space; not available
 * with the random batch list (RBE_ERR_STATE).
 *  skin      > 0: lists at r_list = r_c + skin (length units), rebuilt on the device when
 *            a particle has moved by skin / 2 since the last build; 0: back to cell traversal
 *  capacity  list entries per particle; 0 = automatic: n + 6 sqrt(n) + 32 rounded up to 8,
 *            n = (N / V) 4/3 pi r_list^3 (and the same with N_q for the charged subset's
 *            lists). A longer list sets RBE_ERR_CAPACITY (reported by the next synchronising
 *            call) and its excess entries are dropped.
 * Errors: RBE_ERR_INVALID (skin < 0, not finite, capacity < 0), RBE_ERR_CUTOFF (r_list >= L/2
 * on an axis), RBE_ERR_CELLS (the cell grid cannot hold the build stencil: more than 3
 * cells per side of r_list, or fewer than 2 R + 1 cells on an axis), RBE_ERR_OOM.
 * Forces, energies and neighbour counts are those of the cell traversal (the same exact
 * cutoff decision; FP32 sums in another order). Between builds the particle order is kept,
 * so rbe_get_cells reports the cells of the last build. Discards the captured step graph. */
int rbe_set_neighbor_list(rbe_handle h, double skin, int capacity);

/* List statistics: stats[0] builds and stats[1] force evaluations since the list was
 * enabled, stats[2] / stats[3] longest list of the last build (all particles / charged
 * subset), stats[4] / stats[5] the capacities. Zeros when the list is off. Synchronises. */
int rbe_get_neighbor_list(rbe_handle h, int64_t stats[6]);

/* Throughput probe on the current device, for roofline denominators (it allocates 64
 * bytes of scratch and synchronises the device): kind 0 = FP32 FMA (flop/s, 2 per FMA),
 * 1 = __sincosf pairs per second (the SFU work of one phase of the k-space kernels),
 * 2 = FP64 FMA (flop/s). *ms receives the best kernel time (nullable). */
int rbe_measure_peak(int kind, double *ops_per_s, double *ms);

/* Bytes of device memory held by the handle. */
int rbe_get_memory(rbe_handle h, int64_t *bytes);

/* Checkpoint and resume (the paper does not describe one; the counter-based draws make it
 * exact). rbe_save writes the handle's dynamic state to the file `path`: the step counter,
 * the positions on the 2^-32 grid and the velocities (exact, id order) and the thermostat
 * state, with a fingerprint of the system and parameters. rbe_load reads such a file into a
 * handle created with the same N, box, charges' count, parameters and LJ table
 * (RBE_ERR_STATE otherwise; RBE_ERR_INVALID for an unreadable or malformed file); the next
 * rbe_step or rbe_forces evaluates the forces of the loaded state. Because every mode and
 * random batch draw is a pure function of (seed, replica, step) and the cell order is a pure
 * function of the positions, a run resumed with rbe_load continues bit for bit as the
 * uninterrupted run, with the cell traversal or the random batch list; with a Verlet list the
 * list is rebuilt when needed and forces agree up to FP32 summation order. Both calls
 * synchronise the handle's stream. */
int rbe_save(rbe_handle h, const char *path);
int rbe_load(rbe_handle h, const char *path);

/* Read and clear the device error flags; returns the first of RBE_ERR_SAMPLER,
 * RBE_ERR_NONFINITE, RBE_ERR_CAPACITY that is set, else RBE_OK. Synchronises. */
int rbe_check_device(rbe_handle h);

/* Free every device buffer and the handle. NULL is accepted. */
int rbe_destroy(rbe_handle h);

/* Batched replicas: independent systems of any sizes (each its own rbe_init handle,
 * typically with its own `replica` key) advanced together by one CUDA graph launch per step.
 * Replicas whose Verlet steps launch the same kernels in the same block shapes form a class
 * (same precision, cell traversal, Coulomb arrangement, tuning); every kernel of the step
 * then runs once for the whole class, over the concatenated grids of its replicas, each
 * block reading its replica's own arguments (modes, structure factor, particle arrays) from
 * a table. Results are bit-identical to stepping each replica alone. Classes run as
 * parallel branches of the graph; a replica in no class of two or more (a random batch list
 * or Verlet-list traversal, or a configuration of its own) runs its own step as a branch.
 *  handles  n handles created on the same device; the batch does not own them
 *  cuda_stream  stream the graph is launched on (NULL = legacy default stream)
 * The classes and tables are planned at the first rbe_batch_step (or rbe_batch_info) from
 * the handles' configuration then; change no handle's tuning, traversal or thermostat after.
 * rbe_batch_step is asynchronous; each handle's own getters read its state afterwards
 * (they synchronise the handle's stream, so synchronise cuda_stream first). */
typedef struct rbe_batch_s *rbe_batch;
int rbe_batch_create(rbe_batch *b, int n, const rbe_handle *handles, void *cuda_stream);
int rbe_batch_step(rbe_batch b, int nsteps);
/* The batch plan: number of classes, replicas run by class launches, and kernel launches
 * per batch step (any output may be NULL). Plans the batch if rbe_batch_step has not. */
int rbe_batch_info(rbe_batch b, int32_t *n_classes, int32_t *n_batched, int64_t *kernels);
int rbe_batch_destroy(rbe_batch b);

/* Structure factor rho_l = sum_j q_j exp(2 pi i sum_d m_ld s_jd / 2^32) of N particles for P
 * given modes, computed without allocating any device memory.
 * The paper has no counterpart to this entry point. It exists for callers that cannot
 * allocate device memory: a host application that owns one fixed device pool and forbids
 * libraries to allocate outside it, or a latency-bound loop that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree.
 *  s     device, 3 x N uint32 fractional coordinates, one block per axis (x, then y, then z)
 *  q     device, N float charges
 *  m     device, P x 3 int32 mode integers (row-major)
 *  rho   device, P x 2 double output (Re, Im)
 *  cuda_stream  the stream to run on (NULL = legacy default stream)
 * Sums are Kahan-compensated FP32 per thread, combined in FP64 in a fixed order.
 * Limits: 1 <= P <= 65536 (RBE_ERR_INVALID beyond; nothing is launched then); any N >= 0.
 * The scratch (per-block partial sums) is a fixed 8 MiB device array inside the library,
 * held by every GPU that loads the library until the process exits, and shared by all
 * calls on that GPU: calls that overlap on the GPU race and must be ordered by the
 * caller. The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress) and its SM count; make that first call before any stream capture.
 * The looked-up address is kept for the life of the process, i.e. of the device's primary
 * context: after cudaDeviceReset, or from a thread bound to another (non-primary) context,
 * it is not valid. All pointers and cuda_stream must belong to the device that is current
 * on the calling thread: the array and the launches are taken from that device.
 * Asynchronous: synchronise the stream before reading rho. */
int rbe_structure_factor_noalloc(const uint32_t *s, const float *q, int64_t N,
                                 const int32_t *m, int P, double *rho, void *cuda_stream);

/* Relative half-width of the band around r^2 inside which the kernels take the exact FP64
 * cutoff decision (Eq. Ci_Si: r <= r_c inclusive), for an FP32 r^2 formed from FP32 frame
 * coordinates: each coordinate's magnitude is at most X[d] (Angstrom, X[d] >= 0), the pair
 * is at distance r > 0, the box edges are box[3] > 0, and wrap != 0 when differences are
 * folded into the box. The band is 1.25 times the worst-case rounding bound of that r^2 and
 * never below 1e-5; outside it the FP32 comparison decides exactly. Host-only: needs no GPU
 * and no handle. Returns the band, or -1 for an invalid argument (NULL, non-finite or out
 * of range). */
double rbe_decision_band(const double X[3], double r, const double box[3], int wrap);

/* Static description of an error code. */
const char *rbe_error_string(int code);

/* Library version string. */
const char *rbe_version(void);

#ifdef __cplusplus
}
#endif
#endif
