// rbe_internal.cuh -- device state, helpers and kernel launchers of the RBE force path.
//
// Data layout in HBM (all particle arrays in cell-sorted order, structure of arrays):
//   s[b]      uint32 x 3N   fractional coordinates s_d = r_d / L_d * 2^32 (x block, y, z)
//   vf/vd[b]  velocities (float, or double in the FP64 form), 3N
//   id[b]     int32 N       caller id of the particle at each sorted slot
//   qf/qd[b]  charge (float; double copy in the FP64 form)
//   type[b]   int32 N       LJ type (only when n_types > 1)
//   invm[b]   float N       inverse mass
//   F / Fd    forces in sorted order, 3N
// b in {0,1}: the cell sort writes the other buffer and flips `cur`.
// The charged subset (q != 0) is kept in the same cell order in its own arrays
// (cs, cqf/cqd, cmap: charged slot -> full sorted slot, ccell_start).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/rbe.h"

namespace rbe {

constexpr double kTwo32 = 4294967296.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxTypes = 16;

// Device error bits (OR-ed into ctx.err).
enum : int { ERRBIT_SAMPLER = 1, ERRBIT_NONFINITE = 2, ERRBIT_CAPACITY = 4 };

// Partial-sum slots (doubles per block) of the energy / virial reductions.
enum : int { Q_UREAL = 0, Q_ULJ = 1, Q_WREAL = 2, Q_WLJ = 3, NQ_PAIR = 4 };
constexpr int kCompactMax = 256;  // compacted partials per pair pass before the totals
// Fixed-point scales of the cluster kernel's force sums (64-bit integers): 2^32 in the FP32
// forms, 2^40 in the FP64 form.
constexpr double kFixScale32 = 4294967296.0;
constexpr double kFixScale64 = 1099511627776.0;

struct Grid {
  int n[3];       // cells per axis
  int R[3];       // stencil half-width in cells per axis
  int64_t ncell;
};

struct PairSet {        // one cell-sorted particle set seen by the pair kernels
  const uint32_t *sx, *sy, *sz;
  const float *qf;
  const double *qd;
  const int32_t *type;  // nullptr: single type
  const int32_t *cell_start;
  const int32_t *map;   // output slot of each particle (nullptr: identity)
  int64_t n;
};

// LJ pair coefficients: U = A r^-12 - B r^-6 with A = 4 eps sigma^12, B = 4 eps sigma^6;
// the force factor g (F_i = g (r_i - r_j)) is r^-8 (12 A r^-6 - 6 B), i.e. coefficients
// A12 = 12 A and B6 = 6 B.
struct LJTable {
  float A[kMaxTypes * kMaxTypes], B[kMaxTypes * kMaxTypes];
  float A12[kMaxTypes * kMaxTypes], B6[kMaxTypes * kMaxTypes];
  double Ad[kMaxTypes * kMaxTypes], Bd[kMaxTypes * kMaxTypes];
  double A12d[kMaxTypes * kMaxTypes], B6d[kMaxTypes * kMaxTypes];
  int nt;
};

struct PairConst {
  float h[3];            // L_d / 2^32 (float)
  double hd[3];          // L_d / 2^32 (double)
  float rc2_lo, rc2_hi;  // r_c^2 (1 -/+ band): outside this band FP32 decides
  double rc2d;           // r_c^2, the exact decision inside the band
  float sqrt_alpha, alpha, C;   // Coulomb
  double sqrt_alpha_d, alpha_d, C_d;
  float two_sqrt_alpha_over_sqrt_pi;
  double two_sqrt_alpha_over_sqrt_pi_d;
};

struct Ctx {
  // --- parameters
  int64_t N = 0, Nq = 0;
  double box[3] = {0, 0, 0};
  double alpha = 0, rc = 0, r_core = 0, C = 0, dt = 0, kappa = 0;
  int P = 0, p_rbl = 0, precision = RBE_FP32_COMP, nt = 1, sub = 2;
  bool pair_test16 = true;  // packed half-precision candidate pre-test in the pair kernel
  bool pair_cluster = true;  // cluster-pair kernel (each pair once) for the main pair pass
  bool rbl_eager = false;   // RBL: evaluate every shell pair in the classifying pass
  int rbl_span = 0;         // RBL: group extent in x cells (0: automatic)
  uint64_t seed = 0;
  uint32_t replica = 0;
  bool rbl = false;
  double sum_q2 = 0, U_self = 0, S = 0, V = 0;
  cudaStream_t stream = nullptr;
  int sms = 1;                // SM count of the device the handle was created on
  Grid grid{};
  LJTable lj{};
  void *lj_dev = nullptr;     // device copy of lj (multi-type pair kernels)
  PairConst pc{};
  // --- particle arrays
  int cur = 0;
  uint32_t *s[2] = {nullptr, nullptr};
  float *vf[2] = {nullptr, nullptr};
  double *vd[2] = {nullptr, nullptr};
  int32_t *id[2] = {nullptr, nullptr};
  float *qf[2] = {nullptr, nullptr};
  double *qd[2] = {nullptr, nullptr};
  int32_t *type[2] = {nullptr, nullptr};
  float *invm[2] = {nullptr, nullptr};
  float *F = nullptr;
  double *Fd = nullptr;
  // cluster-pair kernel: fixed-point force sums (3N, sorted order), per-row cluster and
  // super-cluster offsets (rows + 1 each), per-cluster bounds
  long long *facc = nullptr;
  int32_t *cl_base = nullptr, *sc_base = nullptr;
  uint4 *cl_lo = nullptr, *cl_hi = nullptr;
  uint4 *cjrec = nullptr;      // the cluster kernel's j records, 8 slots per cluster, written
                               // with the cluster boxes (FP32 forms)
  uint4 *cq4 = nullptr;        // the same for the charged subset (its Coulomb pass)
  // charged subset
  uint32_t *cs = nullptr;
  float *cqf = nullptr;
  double *cqd = nullptr;
  int32_t *cmap = nullptr;
  // cells
  int32_t *cell_count = nullptr, *ccell_count = nullptr;   // ncell each (contiguous pair)
  int32_t *cell_start = nullptr, *ccell_start = nullptr;   // ncell + 1 each
  int32_t *key = nullptr, *off = nullptr, *tmp = nullptr;  // N each
  int32_t *scan_blk = nullptr;                              // 2 x scan blocks
  int64_t scan_nblk = 0;
  // k-space
  uint64_t *T[3] = {nullptr, nullptr, nullptr};
  int M[3] = {0, 0, 0};
  int4 *m = nullptr;
  float4 *kcf = nullptr;     // (kx, ky, kz, c_l)
  double4_16a *kcd = nullptr;
  double *sf_part = nullptr; // sf blocks x P x 2
  int sf_tile = 256, sf_mb = 128, sf_nblk_p = 0, sf_nblk_m = 0;
  int64_t sf_part_blocks = 0;  // capacity of sf_part in particle blocks
  double2 *rho = nullptr;
  float2 *abf = nullptr;     // (c Im rho, c Re rho)
  double2 *abd = nullptr;
  double *emode = nullptr;   // per-mode (E_l, W_l) pairs: 2P
  // reductions
  double *epart = nullptr;   // partial slots
  double *ecomp = nullptr;   // compacted pair / Coulomb partials [2][kCompactMax][NQ_PAIR]
  int64_t epart_slots = 0;
  int64_t off_pair = 0, off_coul = 0, off_rbl = 0, off_ke = 0, n_pair_blk = 0,
          n_coul_blk = 0, n_rbl_blk = 0, n_ke_blk = 0;
  double *scal = nullptr;    // device scalars (see integrate kernels)
  double *scal_host = nullptr;  // pinned
  uint64_t *step_dev = nullptr;
  uint64_t step = 0;
  int *err = nullptr;
  // debug / outputs
  int32_t *nbr = nullptr;      // sorted order
  int32_t *nshell = nullptr;   // sorted order
  int32_t *partners = nullptr; // sorted order, N x p (ids)
  double *rbl_mean = nullptr;  // 3 doubles: mean short-range force
  double *rbl_part = nullptr;  // RBL blocks x 3
  uint32_t *rbl_masks = nullptr;  // RBL: per slot, warp, chunk and lane: shell masks
  double *rbl_cpart = nullptr;     // RBL: compacted partials (energies NQ_PAIR, then F~ sums 3)
  int *rbl_slots = nullptr;         // RBL: slot pool flags
  int64_t rbl_nslots = 0;
  float *outf = nullptr;       // 3N id-order staging
  double *outd = nullptr;      // 3N id-order staging (FP64 outputs, positions)
  float *out_host = nullptr;   // pinned
  double *pos_stage = nullptr; // 3N doubles (set_positions)
  bool have_forces = false;
  // Nose-Hoover thermostat (NVT); thermo = {xi, eta, s_start, K_end, s_end, xi_end, eta_end}
  bool nvt = false, nvt_primed = false;
  double T0 = 0, tau = 0, kB = 0, Qnh = 0, Nf = 0;
  double *thermo = nullptr;
  // Verlet neighbour list (cell-list real space only): lists warp-interleaved, K entries a
  // particle; vl_flags / vl_count as described in k_list.cu
  bool vl_on = false;
  double vl_skin = 0;
  int vl_K = 0, vl_Kq = 0;
  int vl_R[3] = {0, 0, 0};           // stencil of the build at r_c + skin
  int32_t *vl_list = nullptr, *vl_len = nullptr, *vl_listq = nullptr, *vl_lenq = nullptr;
  uint32_t *vl_ref = nullptr;        // positions at the last build, 3N, sorted order
  uint4 *s4 = nullptr, *cs4 = nullptr;  // packed (s_x, s_y, s_z, q bits): full, charged set
  int32_t *vl_flags = nullptr;       // 8 ints
  unsigned long long *vl_count = nullptr;  // builds, force evaluations
  int64_t vl_bytes = 0;
  // batched replicas: while set, launches are recorded here instead of issued
  struct Recorder *rec = nullptr;
  // graph
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one per starting buffer parity
  cudaGraphExec_t fgraph[2] = {nullptr, nullptr}; // force evaluations (rbe_forces), the same
  cudaStream_t cap_stream = nullptr;  // internal non-blocking stream used only for capture
  cudaStream_t aux_stream = nullptr;  // second capture stream: the k-space branch of a step
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // (fork and join of that branch)
  // profiling: ev[k] is recorded before phase k, ev[RBE_N_PHASE] after the last one
  bool timing = false;
  cudaEvent_t ev[RBE_N_PHASE + 1] = {};
  bool ev_used[RBE_N_PHASE + 1] = {};
  int64_t bytes = 0;
};

// ---------------------------------------------------------------------------------------
// Device helpers

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): two 32x32 products per round,
// multipliers 0xD2511F53 / 0xCD9E8D57, key Weyl increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Cell index along one axis: floor(s * n / 2^32), exact.
__device__ __forceinline__ int cell_of(uint32_t s, int n) {
  return (int)(((uint64_t)s * (uint64_t)n) >> 32);
}

// Phase of exp(i k.r) in turns as a 32-bit fraction: k.r / 2 pi = sum_d m_d s_d / 2^32 (mod 1).
__device__ __forceinline__ uint32_t phase_u32(int4 m, uint32_t sx, uint32_t sy, uint32_t sz) {
  return (uint32_t)m.x * sx + (uint32_t)m.y * sy + (uint32_t)m.z * sz;
}

// Angle in radians in [-pi, pi) of a 32-bit phase, rounded to 2^-23 turns. The rounded
// 23-bit signed value converts to float exactly through the 1.5 * 2^23 bias.
__device__ __forceinline__ float phase_to_radians(uint32_t ph) {
  const int v = ((int)(ph + 256u)) >> 9;  // |v| <= 2^22
  const float f = __int_as_float(0x4B400000 + v) - 12582912.0f;
  return f * (float)(2.0 * kPi / 8388608.0);
}

__device__ __forceinline__ double phase_to_radians_d(uint32_t ph) {
  return (double)(int)ph * (2.0 * kPi / kTwo32);
}

// Add v * scale to a 64-bit fixed-point force sum (round to nearest); an out-of-range value
// sets the non-finite flag instead (its sum would wrap). Integer sums do not depend on the
// order of their terms, so passes that add to the same sums may run in any order.
__device__ __forceinline__ void fx_add(long long *p, float v, float scale, int *err) {
  const float s = v * scale;
  if (fabsf(s) < 4.0e18f) atomicAdd(reinterpret_cast<unsigned long long *>(p),
                                    (unsigned long long)__float2ll_rn(s));
  else atomicOr(err, ERRBIT_NONFINITE);
}
__device__ __forceinline__ void fx_add(long long *p, double v, double scale, int *err) {
  const double s = v * scale;
  if (fabs(s) < 4.0e18) atomicAdd(reinterpret_cast<unsigned long long *>(p),
                                  (unsigned long long)__double2ll_rn(s));
  else atomicOr(err, ERRBIT_NONFINITE);
}
// The same sum for an FP32 v, with the integer nearest s = v * scale built from 32-bit
// conversions: a 64-bit conversion issues to the FP64 pipe, at 1/64 of the FP32 rate, which
// matters in a pass that keeps that pipe busy. |s| < 2^31 converts directly. A larger s is
// an integer (its ulp is at least 2^8) and splits exactly into s = h 2^32 + l with
// h = floor(s 2^-32) and l = s - h 2^32 in [0, 2^32): l is a multiple of s's ulp below 2^32,
// so it has at most 24 significant bits and the FP32 subtraction is exact. The result equals
// the 64-bit conversion's for every |s| < 4e18.
__device__ __forceinline__ void fx_add_i32(long long *p, float v, float scale, int *err) {
  const float s = v * scale;
  if (fabsf(s) < 4.0e18f) {
    const float h = floorf(s * 2.3283064365386963e-10f);
    const unsigned l = __float2uint_rn(s - h * 4294967296.0f);
    const unsigned long long big = ((unsigned long long)(unsigned)__float2int_rn(h) << 32) | l;
    const unsigned long long small = (unsigned long long)(long long)__float2int_rn(s);
    atomicAdd(reinterpret_cast<unsigned long long *>(p), fabsf(s) < 2147483648.0f ? small : big);
  } else {
    atomicOr(err, ERRBIT_NONFINITE);
  }
}
__device__ __forceinline__ void fx_add_i32(long long *p, double v, double scale, int *err) {
  fx_add(p, v, scale, err);
}

// Fused multiply-add a * b + c (one rounding) in either precision. The library is compiled
// without implicit contraction: every fused multiply-add of a kernel is written with these.
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}


// ---------------------------------------------------------------------------------------
// Launches for one replica or for a batch of replicas.
//
// A kernel's work is a body taking its arguments (one struct) and the block's index bx in
// a grid of nbx blocks. The solo kernel runs the body on its own arguments with
// (blockIdx.x, gridDim.x). The batched kernel (suffix _b) runs one launch over the
// concatenated grids of many replicas: replica r owns blocks [pre[r], pre[r+1]) and its own
// argument struct tab[r], so every block does exactly the work of the replica's own launch.
// The library is compiled without implicit multiply-add contraction (every fused
// multiply-add is written out), so the two kernels round every operation alike and give the
// same results bit for bit.

struct BatchIdx {
  int r, bx, nbx;
};

// Replica of this block: the largest r with pre[r] <= blockIdx.x (empty ranges skipped).
__device__ __forceinline__ BatchIdx batch_locate(const int32_t *__restrict__ pre, int nrep) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = nrep;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(pre + mid) <= b) lo = mid; else hi = mid;
  }
  BatchIdx q;
  const int p0 = __ldg(pre + lo);
  q.r = lo;
  q.bx = b - p0;
  q.nbx = __ldg(pre + lo + 1) - p0;
  return q;
}

// One recorded launch: the batched and the solo kernel, whether a batch launches it per
// replica, the replica's grid and block, dynamic shared memory and the bytes of its
// argument struct.
struct RecItem {
  const void *fn, *solo_fn;
  bool per_replica;
  dim3 grid, block;
  size_t smem;
  std::vector<unsigned char> args;
};
struct Recorder {
  std::vector<RecItem> items;
  bool ok = true;  // false: a launch without a batched form was met
};

// Issue the solo kernel on c.stream, or record the launch while c.rec is set. `per_replica`:
// a batch runs this kernel as one solo launch per replica, on parallel branches (the pair
// kernels: their arguments as constant-bank operands save the registers a table costs; a
// batched form of the cluster-pair kernel spilled and ran half as fast again). Otherwise a
// kernel without a batched form (batched == nullptr) makes the recording unusable.
template <class T>
struct NoDeduce {
  using type = T;
};
template <class A>
cudaError_t dispatch(Ctx &c, void (*solo)(A),
                     typename NoDeduce<void (*)(const A *, const int32_t *, int)>::type batched,
                     dim3 grid, dim3 block, size_t smem, const A &a, bool per_replica = false) {
  if (c.rec) {
    if (!batched && !per_replica) {
      c.rec->ok = false;
      return cudaSuccess;
    }
    RecItem it;
    it.fn = reinterpret_cast<const void *>(batched);
    it.solo_fn = reinterpret_cast<const void *>(solo);
    it.per_replica = per_replica;
    it.grid = grid;
    it.block = block;
    it.smem = smem;
    it.args.assign(reinterpret_cast<const unsigned char *>(&a),
                   reinterpret_cast<const unsigned char *>(&a) + sizeof(A));
    c.rec->items.push_back(std::move(it));
    return cudaSuccess;
  }
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  A copy = a;
  void *params[] = {&copy};
  return cudaLaunchKernel(reinterpret_cast<const void *>(solo), grid, block, params, smem, c.stream);
}

// Zero `words` 32-bit words on c.stream (a memset, or a recorded zeroing kernel).
cudaError_t fill_zero(Ctx &c, void *p, int64_t words);

// Solo and batched kernels of a body; LB is the launch-bounds clause, the variadic tail the
// argument type (which may hold template arguments).
#define RBE_KERNELS(LB, NAME, BODY, ...)                                                        \
  __global__ void LB NAME(const __VA_ARGS__ a) { BODY(a, (int)blockIdx.x, (int)gridDim.x); }  \
  __global__ void LB NAME##_b(const __VA_ARGS__ *__restrict__ t,                              \
                              const int32_t *__restrict__ pre, int nrep) {                    \
    const BatchIdx q = batch_locate(pre, nrep);                                               \
    BODY(t[q.r], q.bx, q.nbx);                                                                \
  }
#define RBE_BATCHED_KERNEL(LB, NAME, ARGS, BODY) RBE_KERNELS(LB, NAME, BODY, ARGS)

// ---------------------------------------------------------------------------------------
// Launchers (each in its own translation unit). All return cudaGetLastError().

cudaError_t launch_sample_k(Ctx &c);
cudaError_t launch_bin_sort(Ctx &c);
cudaError_t launch_structure_factor(Ctx &c);
cudaError_t launch_kspace_gather(Ctx &c, bool into_facc);
cudaError_t launch_pair(Ctx &c, bool want_counts);   // per-particle pass, then mark, then Coulomb pass
// Cluster-pair kernel (k_cpair.cu): whether it applies to the handle's box and tuning, the
// launch bounds of its super-clusters and clusters, and the launch (tables, pairs, finish).
bool cpair_usable(const Ctx &c);
int64_t cpair_blocks_bound(const Ctx &c);
int64_t cpair_clusters_bound(const Ctx &c);
cudaError_t launch_cluster_tables(Ctx &c);  // per-row offsets and per-cluster bounds
cudaError_t launch_cluster_pair(Ctx &c, bool coul, bool multi, bool want_counts);
cudaError_t launch_cluster_finish(Ctx &c);
cudaError_t launch_pair_cluster(Ctx &c, bool want_counts);
// Coulomb pass over the charged subset (k_coul.cu): one warp per charged particle; its grid
// (the partial slots of the pass) for nq charged particles.
int64_t coul_blocks(int64_t nq);
cudaError_t launch_coulomb_subset(Ctx &c, const uint4 *s4, bool into_facc);
void mark(Ctx &c, int k);  // record the profiling event k (no-op when profiling is off)
cudaError_t launch_rbl(Ctx &c, bool want_debug);
cudaError_t launch_list_check(Ctx &c);    // rebuild flag from the displacements
cudaError_t launch_list_build(Ctx &c);    // gated list build(s) at r_c + skin
cudaError_t launch_list_commit(Ctx &c);   // gated: reference positions, counters
cudaError_t launch_list_pair(Ctx &c, bool want_counts);  // pair forces from the lists
cudaError_t launch_kick_drift(Ctx &c);  // also advances the device step counter
cudaError_t launch_kick(Ctx &c);
cudaError_t launch_kinetic(Ctx &c);
cudaError_t launch_thermostat(Ctx &c, int mode);  // 0: end + next start half, 1: start half only
cudaError_t launch_totals(Ctx &c);
int64_t partials_compact_count(int64_t nblk);
// The totals sum every slot of a pass's partial range: a pass whose grid writes fewer slots
// than the range holds clears the rest (another kernel may have filled them before).
void zero_partials_tail(Ctx &c, int64_t off, int64_t written, int64_t capacity);
// Relative half-width of the band around r^2 inside which the exact FP64 decision is taken,
// for an FP32 r^2 formed from FP32 frame coordinates with |x_d| <= X[d] (at least 1e-5).
double frame_band(const double X[3], double r, const double box[3], bool wrap);
cudaError_t launch_set_step(Ctx &c, uint64_t step);
cudaError_t launch_step_advance(Ctx &c);
cudaError_t launch_scatter_forces(Ctx &c, bool to_double);
cudaError_t launch_scatter_state(Ctx &c, int what);  // 0: positions, 1: velocities, 2: s
cudaError_t launch_set_positions(Ctx &c);
// Checkpoint load: positions (uint32) and velocities (double), id order, into the sorted slots.
cudaError_t launch_gather_state(Ctx &c, const uint32_t *s_id, const double *v_id);
cudaError_t launch_scatter_int(Ctx &c, const int32_t *src_sorted, int32_t *dst_id, int width);

// Scalars in Ctx::scal (device doubles).
enum : int {
  S_UREAL = 0, S_ULJ, S_UK, S_USELF, S_UTOT, S_KE, S_WREAL, S_WLJ, S_WK, S_WTOT, S_COUNT
};

}  // namespace rbe
