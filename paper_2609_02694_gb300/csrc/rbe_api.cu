// rbe_api.cu -- C ABI of the RBE force path: validation, one-time setup (sampling tables,
// cell grid, device allocation), the force pipeline and the graph-captured Verlet step.
//
// Setup runs once on the host in FP64. The per-axis mode tables follow the sampling
// density of Eq. F_long_RBE, and the cell grid follows the cutoff. Every per-step
// operation runs in the kernels of k_*.cu, on the caller's stream.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "rbe_internal.cuh"

using namespace rbe;

namespace rbe {
int64_t pair_blocks(int64_t n);
int64_t rbl_blocks(int64_t n);
int64_t rbl_slot_count(int64_t n, int sms);
int64_t rbl_compact_count(int64_t nblk);
int64_t rbl_mask_words(int64_t slots);
}  // namespace rbe

struct rbe_ctx : public rbe::Ctx {};

namespace {

#define RBE_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) {                                 \
      fprintf(stderr, "rbe: CUDA error %s at %s:%d\n",       \
              cudaGetErrorString(e_), __FILE__, __LINE__);   \
      return RBE_ERR_CUDA;                                   \
    }                                                        \
  } while (0)

template <typename T>
int dalloc(Ctx &c, T **p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  const size_t bytes = sizeof(T) * (size_t)count;
  if (cudaMalloc((void **)p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return RBE_ERR_OOM;
  }
  c.bytes += (int64_t)bytes;
  return RBE_OK;
}

void dfree(void *p) {
  if (p) cudaFree(p);
}

// Per-axis table of the 1-D discrete Gaussian exp(-k^2 / 4 alpha), k = 2 pi m / L:
// half-width M (weights beyond it are below 2^-53), cumulative thresholds
// T[i] = floor(CDF(m_i) / Z * 2^32) with T[2M] = 2^32, and Z.
int axis_half_width(double L, double alpha) {
  return (int)std::ceil(L * std::sqrt(4.0 * alpha * 53.0 * std::log(2.0)) / (2.0 * kPi));
}

double axis_weight(int m, double L, double alpha) {
  const double km = 2.0 * kPi * (double)m / L;
  return std::exp(-(km * km) / (4.0 * alpha));
}

void axis_table(double L, double alpha, int M, std::vector<uint64_t> &T, double &Z) {
  const int n = 2 * M + 1;
  T.assign(n, 0);
  double z = 0.0;
  for (int i = 0; i < n; ++i) z += axis_weight(i - M, L, alpha);
  double acc = 0.0;
  for (int i = 0; i < n; ++i) {
    acc += axis_weight(i - M, L, alpha);
    T[i] = (uint64_t)std::floor(acc / z * kTwo32);
  }
  T[n - 1] = (uint64_t)1 << 32;
  Z = z;
}

uint32_t quantise(double r, double L) {
  const double f = (r / L) * kTwo32;
  const double fm = f - kTwo32 * std::floor(f / kTwo32);
  return (uint32_t)(unsigned long long)std::llrint(fm);
}

}  // namespace

namespace rbe {
void mark(Ctx &c, int k) {
  if (c.rec || !c.timing || !c.ev[k]) return;
  // during graph capture only an external record becomes an event node of the graph
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c.stream, &st);
  if (st == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(c.ev[k], c.stream, cudaEventRecordExternal);
  else
    cudaEventRecord(c.ev[k], c.stream);
  c.ev_used[k] = true;
}
}  // namespace rbe

namespace {

int free_all(Ctx &c) {
  for (int k = 0; k <= RBE_N_PHASE; ++k)
    if (c.ev[k]) {
      cudaEventDestroy(c.ev[k]);
      c.ev[k] = nullptr;
    }
  for (int b = 0; b < 2; ++b) {
    dfree(c.s[b]); dfree(c.vf[b]); dfree(c.vd[b]); dfree(c.id[b]); dfree(c.qf[b]);
    dfree(c.qd[b]); dfree(c.type[b]); dfree(c.invm[b]);
    if (c.graph[b]) cudaGraphExecDestroy(c.graph[b]);
    c.graph[b] = nullptr;
    if (c.fgraph[b]) cudaGraphExecDestroy(c.fgraph[b]);
    c.fgraph[b] = nullptr;
  }
  dfree(c.F); dfree(c.Fd); dfree(c.facc); dfree(c.cl_base); dfree(c.sc_base); dfree(c.cl_lo);
  dfree(c.cl_hi); dfree(c.cjrec); dfree(c.cq4); dfree(c.cs); dfree(c.cqf); dfree(c.cqd); dfree(c.cmap);
  dfree(c.cell_count); dfree(c.cell_start); dfree(c.key); dfree(c.off); dfree(c.tmp);
  dfree(c.scan_blk);
  for (int d = 0; d < 3; ++d) dfree(c.T[d]);
  dfree(c.m); dfree(c.kcf); dfree(c.kcd); dfree(c.sf_part); dfree(c.rho); dfree(c.abf);
  dfree(c.abd); dfree(c.emode); dfree(c.epart); dfree(c.scal); dfree(c.step_dev);
  dfree(c.err); dfree(c.nbr); dfree(c.ecomp); dfree(c.nshell); dfree(c.partners); dfree(c.rbl_mean);
  dfree(c.rbl_part); dfree(c.rbl_masks); dfree(c.rbl_slots); dfree(c.rbl_cpart); dfree(c.outf); dfree(c.outd); dfree(c.pos_stage); dfree(c.lj_dev);
  dfree(c.thermo);
  dfree(c.vl_list); dfree(c.vl_len); dfree(c.vl_listq); dfree(c.vl_lenq); dfree(c.vl_ref);
  dfree(c.s4); dfree(c.cs4); dfree(c.vl_flags); dfree(c.vl_count);
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  c.cap_stream = nullptr;
  if (c.aux_stream) cudaStreamDestroy(c.aux_stream);
  c.aux_stream = nullptr;
  if (c.ev_fork) cudaEventDestroy(c.ev_fork);
  if (c.ev_join) cudaEventDestroy(c.ev_join);
  c.ev_fork = c.ev_join = nullptr;
  if (c.scal_host) cudaFreeHost(c.scal_host);
  c.scal_host = nullptr;
  return RBE_OK;
}

// The cluster kernel's pipeline in two branches of a captured graph: the k-space chain
// (sampler, structure factor, gather) and the charged subset's Coulomb pass, both into the
// fixed-point sums, on the auxiliary stream beside the cluster tables and the pair pass; then
// the fixed-point finish. The sums are integers, so the forces are those of the sequential
// order bit for bit. The pair pass is issue-bound at three quarters of the issue slots, one
// warp per block; the other branch's kernels fill the slots and SMs it leaves idle (measured
// on 2^20 particles: 1.445 -> 1.360 ms a step, against 1.414 with only the k-space chain
// beside it).
int cluster_pipeline_forked(Ctx &c, bool debug) {
  RBE_CUDA_TRY(cudaEventRecord(c.ev_fork, c.stream));
  RBE_CUDA_TRY(cudaStreamWaitEvent(c.aux_stream, c.ev_fork, 0));
  const cudaStream_t main_stream = c.stream;
  c.stream = c.aux_stream;
  cudaError_t e = launch_sample_k(c);
  if (e == cudaSuccess) e = launch_structure_factor(c);
  if (e == cudaSuccess) e = launch_kspace_gather(c, true);
  const bool fused = c.Nq * 2 > c.N;  // (then the pair pass takes the Coulomb pairs itself)
  if (e == cudaSuccess && !fused) e = launch_coulomb_subset(c, c.cq4, true);
  if (e == cudaSuccess) e = cudaEventRecord(c.ev_join, c.aux_stream);
  c.stream = main_stream;
  RBE_CUDA_TRY(e);
  RBE_CUDA_TRY(launch_cluster_tables(c));
  RBE_CUDA_TRY(launch_cluster_pair(c, fused, c.nt > 1, debug));
  RBE_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.ev_join, 0));
  RBE_CUDA_TRY(launch_cluster_finish(c));
  return RBE_OK;
}

// [list check] -> bin + sort -> sample -> structure factor -> [list build] -> real space
// -> k-space gather (-> the cluster kernel's fixed-point finish)
int force_pipeline(Ctx &c, bool debug) {
  mark(c, RBE_PH_BIN);
  if (c.vl_on) RBE_CUDA_TRY(launch_list_check(c));
  RBE_CUDA_TRY(launch_bin_sort(c));
  const bool cp = !c.rbl && !c.vl_on && cpair_usable(c);
  if (cp && c.Nq > 0 && !c.rec && !c.timing && c.aux_stream) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    RBE_CUDA_TRY(cudaStreamIsCapturing(c.stream, &st));
    if (st == cudaStreamCaptureStatusActive) return cluster_pipeline_forked(c, debug);
  }
  mark(c, RBE_PH_SAMPLE);
  RBE_CUDA_TRY(launch_sample_k(c));
  mark(c, RBE_PH_SF);
  RBE_CUDA_TRY(launch_structure_factor(c));
  mark(c, RBE_PH_LIST);
  if (c.vl_on) {
    RBE_CUDA_TRY(launch_list_build(c));
    RBE_CUDA_TRY(launch_list_commit(c));
  } else if (cp) {
    RBE_CUDA_TRY(launch_cluster_tables(c));  // the cluster-pair kernel's per-step tables
  }
  mark(c, RBE_PH_PAIR);
  if (c.rbl) RBE_CUDA_TRY(launch_rbl(c, debug));
  else if (c.vl_on) RBE_CUDA_TRY(launch_list_pair(c, debug));
  else if (cp) RBE_CUDA_TRY(launch_pair_cluster(c, debug));
  else RBE_CUDA_TRY(launch_pair(c, debug));
  mark(c, RBE_PH_GATHER);
  RBE_CUDA_TRY(launch_kspace_gather(c, cp));
  mark(c, RBE_PH_TAIL);
  if (cp) RBE_CUDA_TRY(launch_cluster_finish(c));
  return RBE_OK;
}

// Kernels one Verlet step launches (memsets excluded).
int64_t kernels_per_step(const Ctx &c) {
  int64_t k = 1;                         // kick-drift (with the step counter)
  k += 6;                                // count, 3 scan passes, scatter, rank+permute
  k += 1;                                // sampler
  k += c.Nq > 0 ? 2 : 0;                 // structure factor + combine
  if (c.rbl) k += 4;                     // RBL, compact partials, mean, subtract
  else k += (c.Nq * 2 > c.N || c.Nq == 0) ? 1 : 2;  // pair passes
  if (!c.rbl && !c.vl_on && cpair_usable(c))
    k += 3;                              // cluster tables (rows, bounds) and the finishing pass
  if (c.vl_on)                           // check, identity copy, build(s), commit
    k += 3 + ((c.Nq * 2 > c.N || c.Nq == 0) ? 1 : 2);
  k += c.Nq > 0 ? 1 : 0;                 // gather
  k += 2;                                // kick (+kinetic), totals
  k += (partials_compact_count(c.n_pair_blk) > 0 ? 1 : 0) +  // partials compaction
       (partials_compact_count(c.n_coul_blk) > 0 ? 1 : 0);
  if (c.nvt) k += 2;                     // thermostat, end-of-step velocity scaling
  return k;
}

int read_device_flags(Ctx &c) {
  int flags = 0;
  RBE_CUDA_TRY(cudaMemcpyAsync(&flags, c.err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  if (flags) {
    RBE_CUDA_TRY(cudaMemsetAsync(c.err, 0, sizeof(int), c.stream));
    if (flags & ERRBIT_SAMPLER) return RBE_ERR_SAMPLER;
    if (flags & ERRBIT_NONFINITE) return RBE_ERR_NONFINITE;
    if (flags & ERRBIT_CAPACITY) return RBE_ERR_CAPACITY;
  }
  return RBE_OK;
}

int copy_scalars(Ctx &c, double *energies, double *virial) {
  RBE_CUDA_TRY(cudaMemcpyAsync(c.scal_host, c.scal, sizeof(double) * S_COUNT,
                               cudaMemcpyDeviceToHost, c.stream));
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  const double *s = c.scal_host;
  if (energies) {
    energies[RBE_E_REAL] = s[S_UREAL];
    energies[RBE_E_LJ] = s[S_ULJ];
    energies[RBE_E_KSPACE] = s[S_UK];
    energies[RBE_E_SELF] = s[S_USELF];
    energies[RBE_E_TOTAL] = s[S_UTOT];
    energies[RBE_E_KINETIC] = s[S_KE];
  }
  if (virial) {
    virial[RBE_W_REAL] = s[S_WREAL];
    virial[RBE_W_LJ] = s[S_WLJ];
    virial[RBE_W_KSPACE] = s[S_WK];
    virial[RBE_W_TOTAL] = s[S_WTOT];
  }
  return RBE_OK;
}

// Capture one Verlet step from buffer parity `parity` into a graph (or, forces_only, one
// force evaluation with the kinetic energy and the totals, as rbe_forces runs it). Capture
// runs on an internal non-blocking stream (the legacy default stream cannot be captured),
// with a second one for the cluster pipeline's other branch; the graph is replayed on
// c.stream.
int capture_step_graph(Ctx &c, int parity, cudaGraphExec_t *out, bool forces_only = false) {
  if (!c.cap_stream) RBE_CUDA_TRY(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
  if (!c.aux_stream) RBE_CUDA_TRY(cudaStreamCreateWithFlags(&c.aux_stream, cudaStreamNonBlocking));
  if (!c.ev_fork) RBE_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
  if (!c.ev_join) RBE_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
  const int saved = c.cur;
  cudaStream_t user = c.stream;
  c.cur = parity;
  c.stream = c.cap_stream;
  cudaGraph_t g = nullptr;
  cudaError_t eb = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
  if (eb != cudaSuccess) {
    c.stream = user;
    c.cur = saved;
    RBE_CUDA_TRY(eb);
  }
  int rc = RBE_OK;
  do {
    if (forces_only) {  // (the step number is set on the device before each launch)
      rc = force_pipeline(c, false);
      if (rc != RBE_OK) break;
      if (launch_kinetic(c) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
      if (launch_totals(c) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
      break;
    }
    mark(c, RBE_PH_KICK_DRIFT);
    if (launch_kick_drift(c) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }  // + step counter
    rc = force_pipeline(c, false);
    if (rc != RBE_OK) break;
    if (launch_kick(c) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
    if (c.nvt && launch_thermostat(c, 0) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
    if (launch_totals(c) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
    mark(c, RBE_N_PHASE);
  } while (0);
  cudaError_t e = cudaStreamEndCapture(c.stream, &g);
  c.cur = saved;
  c.stream = user;
  if (rc != RBE_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  RBE_CUDA_TRY(e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  RBE_CUDA_TRY(e);
  return RBE_OK;
}

}  // namespace

extern "C" {

const char *rbe_version(void) { return "rbe-gb300 1.0 (sm_103a)"; }

double rbe_decision_band(const double X[3], double r, const double box[3], int wrap) {
  if (!X || !box || !(r > 0.0) || !std::isfinite(r)) return -1.0;
  for (int d = 0; d < 3; ++d)
    if (!(X[d] >= 0.0) || !std::isfinite(X[d]) || !(box[d] > 0.0) || !std::isfinite(box[d]))
      return -1.0;
  return frame_band(X, r, box, wrap != 0);
}

const char *rbe_error_string(int code) {
  switch (code) {
    case RBE_OK: return "ok";
    case RBE_ERR_INVALID: return "invalid argument";
    case RBE_ERR_NONNEUTRAL: return "system is not charge neutral";
    case RBE_ERR_CUTOFF: return "cutoff must be smaller than half of every box side";
    case RBE_ERR_CELLS: return "box too small for the cell stencil at this cutoff";
    case RBE_ERR_OOM: return "device allocation failed";
    case RBE_ERR_CUDA: return "CUDA runtime error";
    case RBE_ERR_SAMPLER: return "mode sampler drew k = 0 in 64 consecutive attempts";
    case RBE_ERR_NONFINITE: return "non-finite or runaway position update";
    case RBE_ERR_STATE: return "call not valid in the current state";
    case RBE_ERR_CAPACITY:
      return "neighbour capacity exceeded (RBL stencil over 6144 candidates, or a Verlet "
             "list over its capacity: raise it with rbe_set_neighbor_list)";
    default: return "unknown error";
  }
}

int rbe_init(rbe_handle *hout, const rbe_params *p, int64_t N, const double box[3],
             const double *pos, const double *q, const int32_t *type, const double *mass,
             const double *vel, void *cuda_stream) {
  if (!hout) return RBE_ERR_INVALID;
  *hout = nullptr;
  if (!p || !box || N <= 0 || N >= ((int64_t)1 << 31) || !pos || !q) return RBE_ERR_INVALID;
  if (!(p->alpha > 0) || !(p->r_c > 0) || p->P < 1 || p->P > (1 << 20)) return RBE_ERR_INVALID;
  if (p->precision < RBE_FP32_COMP || p->precision > RBE_FP64) return RBE_ERR_INVALID;
  if (p->n_types < 1 || p->n_types > kMaxTypes || !p->lj_eps || !p->lj_sigma) return RBE_ERR_INVALID;
  if (!(p->coulomb_C >= 0) || !std::isfinite(p->coulomb_C)) return RBE_ERR_INVALID;
  const bool rbl = p->r_core > 0;
  if (rbl && (!(p->r_core < p->r_c) || p->p_rbl < 1 || p->p_rbl > 32)) return RBE_ERR_INVALID;
  if (p->cell_sub < 0 || p->cell_sub > 3) return RBE_ERR_INVALID;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0) || !std::isfinite(box[d])) return RBE_ERR_INVALID;
    if (!(2.0 * p->r_c < box[d])) return RBE_ERR_CUTOFF;
  }
  double qsum = 0.0, qabs = 0.0, q2 = 0.0;
  int64_t Nq = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (!std::isfinite(q[i])) return RBE_ERR_INVALID;
    qsum += q[i];
    qabs += std::fabs(q[i]);
    q2 += q[i] * q[i];
    if (q[i] != 0.0) ++Nq;
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(pos[3 * i + d])) return RBE_ERR_INVALID;
    if (type && (type[i] < 0 || type[i] >= p->n_types)) return RBE_ERR_INVALID;
    if (mass && !(mass[i] > 0)) return RBE_ERR_INVALID;
  }
  if (std::fabs(qsum) > 1e-9 * std::fmax(1.0, qabs)) return RBE_ERR_NONNEUTRAL;

  rbe_ctx *h = new (std::nothrow) rbe_ctx();
  if (!h) return RBE_ERR_OOM;
  Ctx &c = *h;
  c.N = N; c.Nq = Nq;
  for (int d = 0; d < 3; ++d) c.box[d] = box[d];
  c.V = box[0] * box[1] * box[2];
  c.alpha = p->alpha; c.rc = p->r_c; c.r_core = rbl ? p->r_core : 0.0;
  c.C = p->coulomb_C; c.dt = p->dt; c.kappa = p->kappa;
  c.P = p->P; c.p_rbl = rbl ? p->p_rbl : 0; c.precision = p->precision;
  // the cluster kernel evaluates about a quarter more candidate pairs than the per-particle
  // kernel: cheaper in FP32, where its per-pair overhead is saved, not in the FP64 form
  c.pair_cluster = p->precision != RBE_FP64;
  c.nt = p->n_types; c.seed = p->seed; c.replica = p->replica; c.rbl = rbl;
  c.stream = (cudaStream_t)cuda_stream;
  c.sum_q2 = q2;
  c.U_self = c.C * std::sqrt(c.alpha / kPi) * q2;
  if (rbl) {  // eager shell evaluation when the mean shell holds no more than p particles
    const double vol = box[0] * box[1] * box[2];
    const double shell_mean = (double)N / vol * (4.0 / 3.0) * kPi *
                              (c.rc * c.rc * c.rc - c.r_core * c.r_core * c.r_core);
    c.rbl_eager = shell_mean <= (double)c.p_rbl;
  }

  // cell grid
  if (rbl) {
    c.sub = 1;
    for (int d = 0; d < 3; ++d) {
      c.grid.n[d] = (int)std::floor(box[d] / c.rc);
      c.grid.R[d] = 1;
      if (c.grid.n[d] < 3) { delete h; return RBE_ERR_CELLS; }
    }
  } else {
    int sub = p->cell_sub > 0 ? p->cell_sub : 2;
    for (;; --sub) {
      bool ok = true;
      for (int d = 0; d < 3; ++d) {
        c.grid.n[d] = (int)std::floor(box[d] * sub / c.rc);
        const double a = box[d] / c.grid.n[d];
        c.grid.R[d] = (int)std::ceil(c.rc / a);
        if (c.grid.n[d] < 2 * c.grid.R[d] + 1) ok = false;
      }
      if (ok) break;
      if (sub == 1) { delete h; return RBE_ERR_CELLS; }
    }
    c.sub = sub;
  }
  c.grid.ncell = (int64_t)c.grid.n[0] * c.grid.n[1] * c.grid.n[2];
  if (c.grid.ncell >= ((int64_t)1 << 31) - 2) { delete h; return RBE_ERR_CELLS; }

  // pair constants
  for (int d = 0; d < 3; ++d) {
    c.pc.hd[d] = box[d] / kTwo32;
    c.pc.h[d] = (float)c.pc.hd[d];
  }
  const double rc2 = c.rc * c.rc;
  c.pc.rc2d = rc2;
  c.pc.rc2_lo = (float)(rc2 * (1.0 - 1e-5));
  c.pc.rc2_hi = (float)(rc2 * (1.0 + 1e-5));
  c.pc.alpha_d = c.alpha; c.pc.alpha = (float)c.alpha;
  c.pc.sqrt_alpha_d = std::sqrt(c.alpha); c.pc.sqrt_alpha = (float)c.pc.sqrt_alpha_d;
  c.pc.C_d = c.C; c.pc.C = (float)c.C;
  c.pc.two_sqrt_alpha_over_sqrt_pi_d = 2.0 * std::sqrt(c.alpha) / std::sqrt(kPi);
  c.pc.two_sqrt_alpha_over_sqrt_pi = (float)c.pc.two_sqrt_alpha_over_sqrt_pi_d;
  // LJ table
  c.lj.nt = c.nt;
  for (int a = 0; a < c.nt; ++a)
    for (int b = 0; b < c.nt; ++b) {
      const int k = a * c.nt + b;
      const double e = p->lj_eps[k], s = p->lj_sigma[k];
      if (!(e >= 0) || !(s > 0) || p->lj_eps[b * c.nt + a] != e || p->lj_sigma[b * c.nt + a] != s) {
        delete h;
        return RBE_ERR_INVALID;
      }
      const double s6 = (s * s) * (s * s) * (s * s), s12 = s6 * s6;
      c.lj.Ad[k] = 4.0 * e * s12; c.lj.Bd[k] = 4.0 * e * s6;
      c.lj.A12d[k] = 48.0 * e * s12; c.lj.B6d[k] = 24.0 * e * s6;
      c.lj.A[k] = (float)c.lj.Ad[k]; c.lj.B[k] = (float)c.lj.Bd[k];
      c.lj.A12[k] = (float)c.lj.A12d[k]; c.lj.B6[k] = (float)c.lj.B6d[k];
    }

  // sampling tables
  std::vector<uint64_t> T[3];
  double Z[3];
  for (int d = 0; d < 3; ++d) {
    c.M[d] = axis_half_width(box[d], c.alpha);
    axis_table(box[d], c.alpha, c.M[d], T[d], Z[d]);
  }
  c.S = Z[0] * Z[1] * Z[2] - 1.0;

  // SM count of the current device (for the launch shapes below)
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      delete h;
      return RBE_ERR_CUDA;
    }
    c.sms = sms;
  }
  // structure-factor launch shape: one thread per mode, particle tiles per block
  c.sf_mb = std::min(256, ((c.P + 31) / 32) * 32);
  c.sf_nblk_m = (c.P + c.sf_mb - 1) / c.sf_mb;
  {
    const int64_t target_blocks = (int64_t)c.sms * 8;
    int64_t tile = Nq * c.sf_nblk_m / std::max<int64_t>(1, target_blocks);
    tile = std::max<int64_t>(32, std::min<int64_t>(512, ((tile + 31) / 32) * 32));
    c.sf_tile = (int)tile;
    c.sf_nblk_p = (int)std::max<int64_t>(1, (Nq + tile - 1) / tile);
    c.sf_part_blocks = std::max<int64_t>(1, (Nq + 31) / 32);  // room for the smallest tile
  }

  // reductions layout
  c.n_pair_blk = rbl ? 0 : std::max(pair_blocks(N), cpair_blocks_bound(c));
  c.n_coul_blk = rbl ? 0 : std::max(pair_blocks(Nq), coul_blocks(Nq));
  c.n_rbl_blk = rbl ? rbl_blocks(N) : 0;
  c.rbl_nslots = rbl ? rbl_slot_count(N, c.sms) : 0;
  c.n_ke_blk = (N + 255) / 256;
  c.off_pair = 0;
  c.off_coul = c.off_pair + c.n_pair_blk * NQ_PAIR;
  c.off_rbl = c.off_coul + c.n_coul_blk * NQ_PAIR;
  c.off_ke = c.off_rbl + c.n_rbl_blk * NQ_PAIR;
  c.epart_slots = c.off_ke + c.n_ke_blk;
  c.scan_nblk = (c.grid.ncell + 2047) / 2048;

  // allocation
  const bool fp64 = c.precision == RBE_FP64;
  int rc = RBE_OK;
  for (int b = 0; b < 2 && rc == RBE_OK; ++b) {
    rc |= dalloc(c, &c.s[b], 3 * N);
    if (fp64) rc |= dalloc(c, &c.vd[b], 3 * N);
    else rc |= dalloc(c, &c.vf[b], 3 * N);
    rc |= dalloc(c, &c.id[b], N);
    rc |= dalloc(c, &c.qf[b], N);
    if (fp64) rc |= dalloc(c, &c.qd[b], N);
    if (c.nt > 1) rc |= dalloc(c, &c.type[b], N);
    rc |= dalloc(c, &c.invm[b], N);
  }
  if (fp64) rc |= dalloc(c, &c.Fd, 3 * N);
  else rc |= dalloc(c, &c.F, 3 * N);
  if (!rbl) {
    const int64_t nrows = (int64_t)c.grid.n[1] * c.grid.n[2];
    rc |= dalloc(c, &c.facc, 3 * N);
    rc |= dalloc(c, &c.cl_base, nrows + 1);
    rc |= dalloc(c, &c.sc_base, nrows + 1);
    rc |= dalloc(c, &c.cl_lo, cpair_clusters_bound(c));
    rc |= dalloc(c, &c.cl_hi, cpair_clusters_bound(c));
    if (!fp64) rc |= dalloc(c, &c.cjrec, 8 * cpair_clusters_bound(c));  // 8 slots per cluster
    rc |= dalloc(c, &c.cq4, Nq);
  }
  rc |= dalloc(c, &c.cs, 3 * Nq);
  rc |= dalloc(c, &c.cqf, Nq);
  if (fp64) rc |= dalloc(c, &c.cqd, Nq);
  rc |= dalloc(c, &c.cmap, Nq);
  rc |= dalloc(c, &c.cell_count, 2 * c.grid.ncell);
  rc |= dalloc(c, &c.cell_start, 2 * (c.grid.ncell + 1));
  rc |= dalloc(c, &c.key, N);
  rc |= dalloc(c, &c.off, N);
  rc |= dalloc(c, &c.tmp, N);
  rc |= dalloc(c, &c.scan_blk, 2 * c.scan_nblk);
  for (int d = 0; d < 3; ++d) rc |= dalloc(c, &c.T[d], 2 * c.M[d] + 1);
  rc |= dalloc(c, &c.m, c.P);
  rc |= dalloc(c, &c.kcf, c.P);
  rc |= dalloc(c, &c.kcd, c.P);
  rc |= dalloc(c, &c.sf_part, c.sf_part_blocks * c.P * 2);
  rc |= dalloc(c, &c.rho, c.P);
  rc |= dalloc(c, &c.abf, c.P);
  rc |= dalloc(c, &c.abd, c.P);
  rc |= dalloc(c, &c.emode, 2 * c.P);
  rc |= dalloc(c, &c.epart, c.epart_slots);
  rc |= dalloc(c, &c.ecomp, 2 * kCompactMax * NQ_PAIR);
  rc |= dalloc(c, &c.scal, S_COUNT);
  rc |= dalloc(c, &c.step_dev, 1);
  rc |= dalloc(c, &c.err, 1);
  rc |= dalloc(c, &c.nbr, N);
  if (rbl) {
    rc |= dalloc(c, &c.nshell, N);
    rc |= dalloc(c, &c.partners, N * c.p_rbl);
    rc |= dalloc(c, &c.rbl_part, c.n_rbl_blk * 3);
    rc |= dalloc(c, &c.rbl_masks, rbl_mask_words(c.rbl_nslots));
    rc |= dalloc(c, &c.rbl_slots, c.rbl_nslots);
    rc |= dalloc(c, &c.rbl_cpart, rbl_compact_count(c.n_rbl_blk) * (NQ_PAIR + 3));
  }
  rc |= dalloc(c, &c.rbl_mean, 3);
  rc |= dalloc(c, &c.outf, 3 * N);
  rc |= dalloc(c, &c.outd, 3 * N);
  rc |= dalloc(c, &c.pos_stage, 3 * N);
  rc |= dalloc(c, reinterpret_cast<char **>(&c.lj_dev), (int64_t)sizeof(LJTable));
  if (rc != RBE_OK) {
    free_all(c);
    delete h;
    return RBE_ERR_OOM;
  }
  if (cudaMallocHost((void **)&c.scal_host, sizeof(double) * S_COUNT) != cudaSuccess) {
    cudaGetLastError();
    free_all(c);
    delete h;
    return RBE_ERR_OOM;
  }
  c.cell_start += 0;
  c.ccell_start = c.cell_start + (c.grid.ncell + 1);
  c.ccell_count = c.cell_count + c.grid.ncell;

  // initial state (identity order), uploaded once
  {
    std::vector<uint32_t> s(3 * N);
    std::vector<int32_t> ids(N), ty;
    std::vector<float> qf(N), im(N), vf;
    std::vector<double> vd;
    for (int64_t i = 0; i < N; ++i) {
      for (int d = 0; d < 3; ++d) s[d * N + i] = quantise(pos[3 * i + d], box[d]);
      ids[i] = (int32_t)i;
      qf[i] = (float)q[i];
      im[i] = (float)(1.0 / (mass ? mass[i] : 1.0));
    }
    int e = 0;
    e |= cudaMemcpy(c.s[0], s.data(), sizeof(uint32_t) * 3 * N, cudaMemcpyHostToDevice);
    e |= cudaMemcpy(c.id[0], ids.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice);
    e |= cudaMemcpy(c.qf[0], qf.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    e |= cudaMemcpy(c.invm[0], im.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    if (fp64) e |= cudaMemcpy(c.qd[0], q, sizeof(double) * N, cudaMemcpyHostToDevice);
    if (c.nt > 1) {
      ty.assign(N, 0);
      if (type) for (int64_t i = 0; i < N; ++i) ty[i] = type[i];
      e |= cudaMemcpy(c.type[0], ty.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice);
    }
    if (fp64) {
      vd.assign(3 * N, 0.0);
      if (vel) for (int64_t i = 0; i < N; ++i) for (int d = 0; d < 3; ++d) vd[d * N + i] = vel[3 * i + d];
      e |= cudaMemcpy(c.vd[0], vd.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice);
    } else {
      vf.assign(3 * N, 0.f);
      if (vel) for (int64_t i = 0; i < N; ++i) for (int d = 0; d < 3; ++d) vf[d * N + i] = (float)vel[3 * i + d];
      e |= cudaMemcpy(c.vf[0], vf.data(), sizeof(float) * 3 * N, cudaMemcpyHostToDevice);
    }
    for (int d = 0; d < 3; ++d)
      e |= cudaMemcpy(c.T[d], T[d].data(), sizeof(uint64_t) * T[d].size(), cudaMemcpyHostToDevice);
    e |= cudaMemcpy(c.lj_dev, &c.lj, sizeof(LJTable), cudaMemcpyHostToDevice);
    e |= cudaMemset(c.epart, 0, sizeof(double) * c.epart_slots);
    e |= cudaMemset(c.emode, 0, sizeof(double) * 2 * c.P);
    e |= cudaMemset(c.err, 0, sizeof(int));
    if (c.facc) e |= cudaMemset(c.facc, 0, sizeof(long long) * 3 * N);
    if (c.rbl_slots) e |= cudaMemset(c.rbl_slots, 0, sizeof(int) * c.rbl_nslots);
    e |= cudaMemset(c.step_dev, 0, sizeof(uint64_t));
    e |= cudaMemset(c.scal, 0, sizeof(double) * S_COUNT);
    if (e != 0) {
      cudaGetLastError();
      free_all(c);
      delete h;
      return RBE_ERR_CUDA;
    }
  }
  *hout = h;
  return RBE_OK;
}

int rbe_destroy(rbe_handle h) {
  if (!h) return RBE_OK;
  cudaStreamSynchronize(h->stream);
  free_all(*h);
  delete h;
  return RBE_OK;
}

int rbe_sample_k(rbe_handle h, uint64_t step, int32_t *m_out, double *S_out) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  RBE_CUDA_TRY(launch_set_step(c, step));
  RBE_CUDA_TRY(launch_sample_k(c));
  c.have_forces = false;
  if (m_out) {
    std::vector<int4> mm(c.P);
    RBE_CUDA_TRY(cudaMemcpyAsync(mm.data(), c.m, sizeof(int4) * c.P, cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    for (int l = 0; l < c.P; ++l) {
      m_out[3 * l] = mm[l].x; m_out[3 * l + 1] = mm[l].y; m_out[3 * l + 2] = mm[l].z;
    }
  }
  if (S_out) *S_out = c.S;
  return read_device_flags(c);
}

int rbe_set_positions(rbe_handle h, const double *pos, int on_device) {
  if (!h || !pos) return RBE_ERR_INVALID;
  Ctx &c = *h;
  RBE_CUDA_TRY(cudaMemcpyAsync(c.pos_stage, pos, sizeof(double) * 3 * c.N,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               c.stream));
  // (a Verlet list stays valid: new positions are written in the kept order, and the next
  //  displacement check against the build positions decides whether to rebuild)
  RBE_CUDA_TRY(launch_set_positions(c));
  c.have_forces = false;
  return RBE_OK;
}

static int forces_common(rbe_handle h, uint64_t step, bool debug) {
  Ctx &c = *h;
  RBE_CUDA_TRY(launch_set_step(c, step));
  if (!debug && !c.timing) {
    // replay a captured evaluation (one graph per buffer parity, as for rbe_step)
    if (!c.fgraph[c.cur]) {
      const int rc = capture_step_graph(c, c.cur, &c.fgraph[c.cur], true);
      if (rc != RBE_OK) return rc;
    }
    RBE_CUDA_TRY(cudaGraphLaunch(c.fgraph[c.cur], c.stream));
    c.cur = 1 - c.cur;
    c.have_forces = (step == c.step);
    return RBE_OK;
  }
  mark(c, RBE_PH_KICK_DRIFT);
  int rc = force_pipeline(c, debug);
  if (rc != RBE_OK) return rc;
  RBE_CUDA_TRY(launch_kinetic(c));
  RBE_CUDA_TRY(launch_totals(c));
  mark(c, RBE_N_PHASE);
  c.have_forces = (step == c.step);
  return RBE_OK;
}

int rbe_forces(rbe_handle h, uint64_t step, float *F_out, int F_on_device, double *energies,
               double *virial) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  int rc = forces_common(h, step, false);  // no neighbour counts or RBL partners
  if (rc != RBE_OK) return rc;
  if (F_out) {
    RBE_CUDA_TRY(launch_scatter_forces(c, false));
    RBE_CUDA_TRY(cudaMemcpyAsync(F_out, c.outf, sizeof(float) * 3 * c.N,
                                 F_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c.stream));
  }
  if (energies || virial) {
    rc = copy_scalars(c, energies, virial);
    if (rc != RBE_OK) return rc;
  }
  if ((F_out && !F_on_device) || energies || virial) return read_device_flags(c);
  return RBE_OK;
}

int rbe_forces_f64(rbe_handle h, uint64_t step, double *F_out, double *energies, double *virial) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  int rc = forces_common(h, step, true);
  if (rc != RBE_OK) return rc;
  if (F_out) {
    RBE_CUDA_TRY(launch_scatter_forces(c, true));
    RBE_CUDA_TRY(cudaMemcpyAsync(F_out, c.outd, sizeof(double) * 3 * c.N, cudaMemcpyDeviceToHost,
                                 c.stream));
  }
  rc = copy_scalars(c, energies, virial);
  if (rc != RBE_OK) return rc;
  return read_device_flags(c);
}

int rbe_step(rbe_handle h, int nsteps) {
  if (!h || nsteps < 0) return RBE_ERR_INVALID;
  Ctx &c = *h;
  if (nsteps == 0) return RBE_OK;
  if (!c.have_forces) {
    int rc = forces_common(h, c.step, false);
    if (rc != RBE_OK) return rc;
  }
  if (c.nvt && !c.nvt_primed) {  // start half of the first thermostatted step
    RBE_CUDA_TRY(launch_kinetic(c));
    RBE_CUDA_TRY(launch_thermostat(c, 1));
    c.nvt_primed = true;
  }
  for (int b = 0; b < 2; ++b)
    if (!c.graph[b]) {
      int rc = capture_step_graph(c, b, &c.graph[b]);
      if (rc != RBE_OK) return rc;
    }
  for (int k = 0; k < nsteps; ++k) {
    RBE_CUDA_TRY(cudaGraphLaunch(c.graph[c.cur], c.stream));
    c.cur = 1 - c.cur;
    c.step += 1;
  }
  c.have_forces = true;
  return RBE_OK;
}

static void drop_graphs(Ctx &c);

int rbe_set_thermostat(rbe_handle h, double T_target, double tau, double kB) {
  if (!h || !std::isfinite(T_target) || !std::isfinite(tau) || !std::isfinite(kB))
    return RBE_ERR_INVALID;
  Ctx &c = *h;
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  const bool on = tau > 0;
  if (on && (!(T_target > 0) || !(kB > 0) || c.N < 2)) return RBE_ERR_INVALID;
  if (!c.thermo && dalloc(c, &c.thermo, 7) != RBE_OK) return RBE_ERR_OOM;
  const double init[7] = {0.0, 0.0, 1.0, 0.0, 1.0, 0.0, 0.0};
  RBE_CUDA_TRY(cudaMemcpy(c.thermo, init, sizeof(init), cudaMemcpyHostToDevice));
  c.nvt = on;
  c.nvt_primed = false;
  c.T0 = T_target; c.tau = tau; c.kB = kB;
  c.Nf = 3.0 * (double)c.N - 3.0;
  c.Qnh = c.Nf * kB * T_target * tau * tau;
  drop_graphs(c);
  return RBE_OK;
}

int rbe_get_thermostat(rbe_handle h, double out[3]) {
  if (!h || !out) return RBE_ERR_INVALID;
  Ctx &c = *h;
  double th[7] = {0.0, 0.0, 1.0, 0.0, 1.0, 0.0, 0.0};
  if (c.thermo) {
    RBE_CUDA_TRY(cudaMemcpyAsync(th, c.thermo, sizeof(th), cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  }
  // xi and eta at the end of the last step (the device copy already holds the next step's
  // start half, whose velocity scaling is still pending)
  out[0] = th[5];
  out[1] = th[6];
  out[2] = c.nvt ? 0.5 * c.Qnh * th[5] * th[5] + c.Nf * c.kB * c.T0 * th[6] : 0.0;
  return RBE_OK;
}

int rbe_get_step(rbe_handle h, uint64_t *step) {
  if (!h || !step) return RBE_ERR_INVALID;
  *step = h->step;
  return RBE_OK;
}

int rbe_get_energies(rbe_handle h, double *energies, double *virial) {
  if (!h) return RBE_ERR_INVALID;
  return copy_scalars(*h, energies, virial);
}

int rbe_get_state(rbe_handle h, double *pos, double *vel, uint32_t *s_frac) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  if (pos) {
    RBE_CUDA_TRY(launch_scatter_state(c, 0));
    RBE_CUDA_TRY(cudaMemcpyAsync(pos, c.outd, sizeof(double) * 3 * c.N, cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  }
  if (vel) {
    RBE_CUDA_TRY(launch_scatter_state(c, 1));
    RBE_CUDA_TRY(cudaMemcpyAsync(vel, c.outd, sizeof(double) * 3 * c.N, cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  }
  if (s_frac) {
    RBE_CUDA_TRY(launch_scatter_state(c, 2));
    RBE_CUDA_TRY(cudaMemcpyAsync(s_frac, c.outf, sizeof(uint32_t) * 3 * c.N, cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  }
  return read_device_flags(c);
}

int rbe_get_cells(rbe_handle h, int32_t n_cells[3], int64_t *cell_start, int64_t *sorted_ids) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  if (n_cells) for (int d = 0; d < 3; ++d) n_cells[d] = c.grid.n[d];
  if (cell_start) {
    std::vector<int32_t> cs(c.grid.ncell + 1);
    RBE_CUDA_TRY(cudaMemcpyAsync(cs.data(), c.cell_start, sizeof(int32_t) * cs.size(),
                                 cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    for (size_t k = 0; k < cs.size(); ++k) cell_start[k] = cs[k];
  }
  if (sorted_ids) {
    std::vector<int32_t> ids(c.N);
    RBE_CUDA_TRY(cudaMemcpyAsync(ids.data(), c.id[c.cur], sizeof(int32_t) * c.N,
                                 cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    for (int64_t k = 0; k < c.N; ++k) sorted_ids[k] = ids[k];
  }
  return RBE_OK;
}

int rbe_get_rho(rbe_handle h, double *rho, int32_t *m_out) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  if (rho) {
    RBE_CUDA_TRY(cudaMemcpyAsync(rho, c.rho, sizeof(double2) * c.P, cudaMemcpyDeviceToHost, c.stream));
  }
  if (m_out) {
    std::vector<int4> mm(c.P);
    RBE_CUDA_TRY(cudaMemcpyAsync(mm.data(), c.m, sizeof(int4) * c.P, cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    for (int l = 0; l < c.P; ++l) {
      m_out[3 * l] = mm[l].x; m_out[3 * l + 1] = mm[l].y; m_out[3 * l + 2] = mm[l].z;
    }
  }
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return RBE_OK;
}

int rbe_get_neighbor_counts(rbe_handle h, int32_t *n_core, int32_t *n_shell) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  int32_t *dst = reinterpret_cast<int32_t *>(c.outf);
  if (n_core) {
    RBE_CUDA_TRY(launch_scatter_int(c, c.nbr, dst, 1));
    RBE_CUDA_TRY(cudaMemcpyAsync(n_core, dst, sizeof(int32_t) * c.N, cudaMemcpyDeviceToHost, c.stream));
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  }
  if (n_shell) {
    if (c.rbl) {
      RBE_CUDA_TRY(launch_scatter_int(c, c.nshell, dst, 1));
      RBE_CUDA_TRY(cudaMemcpyAsync(n_shell, dst, sizeof(int32_t) * c.N, cudaMemcpyDeviceToHost, c.stream));
      RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    } else {
      memset(n_shell, 0, sizeof(int32_t) * c.N);
    }
  }
  return RBE_OK;
}

int rbe_get_rbl_partners(rbe_handle h, int32_t *partners) {
  if (!h || !partners) return RBE_ERR_INVALID;
  Ctx &c = *h;
  if (!c.rbl) return RBE_ERR_STATE;
  std::vector<int32_t> srt((size_t)c.N * c.p_rbl), ids(c.N);
  RBE_CUDA_TRY(cudaMemcpyAsync(srt.data(), c.partners, sizeof(int32_t) * srt.size(),
                               cudaMemcpyDeviceToHost, c.stream));
  RBE_CUDA_TRY(cudaMemcpyAsync(ids.data(), c.id[c.cur], sizeof(int32_t) * c.N,
                               cudaMemcpyDeviceToHost, c.stream));
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  for (int64_t k = 0; k < c.N; ++k)
    memcpy(partners + (size_t)ids[k] * c.p_rbl, srt.data() + (size_t)k * c.p_rbl,
           sizeof(int32_t) * c.p_rbl);
  return RBE_OK;
}

int rbe_set_profiling(rbe_handle h, int enable) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  const bool on = enable != 0;
  if (on == c.timing) return RBE_OK;
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  drop_graphs(c);  // (steps and force evaluations are captured again, with or without events)
  if (on)
    for (int k = 0; k <= RBE_N_PHASE; ++k)
      if (!c.ev[k]) RBE_CUDA_TRY(cudaEventCreate(&c.ev[k]));
  c.timing = on;
  return RBE_OK;
}

int rbe_get_profile(rbe_handle h, double *phase_ms, int64_t *kps) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  if (kps) *kps = kernels_per_step(c);
  if (phase_ms) {
    if (!c.timing) return RBE_ERR_STATE;
    RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    for (int k = 0; k < RBE_N_PHASE; ++k) {
      float ms = 0.f;
      // a phase that was not recorded in the last run (e.g. no kick-drift in rbe_forces)
      // reads as zero
      if (c.ev_used[k] && c.ev_used[k + 1]) {
        if (cudaEventElapsedTime(&ms, c.ev[k], c.ev[k + 1]) != cudaSuccess) {
          cudaGetLastError();
          ms = 0.f;
        }
      }
      phase_ms[k] = ms;
    }
  }
  return RBE_OK;
}

static void drop_graphs(Ctx &c) {
  for (int b = 0; b < 2; ++b) {
    if (c.graph[b]) {
      cudaGraphExecDestroy(c.graph[b]);
      c.graph[b] = nullptr;
    }
    if (c.fgraph[b]) {
      cudaGraphExecDestroy(c.fgraph[b]);
      c.fgraph[b] = nullptr;
    }
  }
}

// Structure-factor launch shape for a tile of `tile` particles per block.
static void set_sf_tile(Ctx &c, int64_t tile) {
  c.sf_tile = (int)tile;
  c.sf_nblk_p = (int)std::max<int64_t>(1, (c.Nq + tile - 1) / tile);
}

int rbe_set_tuning(rbe_handle h, int key, int value) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  if (key == RBE_TUNE_PAIR_TEST16) {
    if (value != 0 && value != 1) return RBE_ERR_INVALID;
    c.pair_test16 = value != 0;
  } else if (key == RBE_TUNE_PAIR_CLUSTER) {
    if (value != 0 && value != 1) return RBE_ERR_INVALID;
    c.pair_cluster = value != 0;
  } else if (key == RBE_TUNE_RBL_EAGER) {
    if (value != 0 && value != 1) return RBE_ERR_INVALID;
    c.rbl_eager = value != 0;
  } else if (key == RBE_TUNE_RBL_SPAN) {
    if (value < 0 || value > 14) return RBE_ERR_INVALID;
    c.rbl_span = value;
  } else if (key == RBE_TUNE_SF_TILE) {
    if (value < 32 || value > 1024 || value % 32) return RBE_ERR_INVALID;
    // the partial buffer was sized for the initial tile; smaller tiles need more blocks
    const int64_t nblk = std::max<int64_t>(1, (c.Nq + value - 1) / value);
    if (nblk > c.sf_part_blocks) return RBE_ERR_INVALID;
    set_sf_tile(c, value);
  } else {
    return RBE_ERR_INVALID;
  }
  drop_graphs(c);
  return RBE_OK;
}

int rbe_get_tuning(rbe_handle h, int key, int *value) {
  if (!h || !value) return RBE_ERR_INVALID;
  if (key == RBE_TUNE_PAIR_TEST16) *value = h->pair_test16 ? 1 : 0;
  else if (key == RBE_TUNE_SF_TILE) *value = h->sf_tile;
  else if (key == RBE_TUNE_RBL_EAGER) *value = h->rbl_eager ? 1 : 0;
  else if (key == RBE_TUNE_RBL_SPAN) *value = h->rbl_span;
  else if (key == RBE_TUNE_PAIR_CLUSTER) *value = h->pair_cluster ? 1 : 0;
  else return RBE_ERR_INVALID;
  return RBE_OK;
}

static int time_forces(Ctx &c, int reps, float *ms_out) {
  cudaEvent_t e0, e1;
  RBE_CUDA_TRY(cudaEventCreate(&e0));
  RBE_CUDA_TRY(cudaEventCreate(&e1));
  int rc = force_pipeline(c, false);  // warm
  RBE_CUDA_TRY(cudaEventRecord(e0, c.stream));
  for (int r = 0; r < reps && rc == RBE_OK; ++r) rc = force_pipeline(c, false);
  RBE_CUDA_TRY(cudaEventRecord(e1, c.stream));
  RBE_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms;
  return rc;
}

int rbe_autotune(rbe_handle h, int reps, int *chosen) {
  if (!h || reps < 1) return RBE_ERR_INVALID;
  Ctx &c = *h;
  const bool saved_timing = c.timing;
  c.timing = false;
  RBE_CUDA_TRY(launch_set_step(c, c.step));
  float best = 0.f;
  int best16 = c.pair_test16 ? 1 : 0;
  // the per-particle kernel's two pre-tests, then the cluster-pair kernel against the better
  const bool cl_saved = c.pair_cluster;
  c.pair_cluster = false;
  for (int v = 0; v <= 1; ++v) {
    c.pair_test16 = v != 0;
    float ms = 0.f;
    int rc = time_forces(c, reps, &ms);
    if (rc != RBE_OK) { c.timing = saved_timing; c.pair_cluster = cl_saved; return rc; }
    if (v == 0 || ms < best) { best = ms; best16 = v; }
  }
  c.pair_test16 = best16 != 0;
  int best_cl = 0;
  if (!c.rbl) {
    c.pair_cluster = true;
    if (cpair_usable(c)) {
      float ms = 0.f;
      int rc = time_forces(c, reps, &ms);
      if (rc != RBE_OK) { c.timing = saved_timing; return rc; }
      if (ms < best) { best = ms; best_cl = 1; }
    }
    c.pair_cluster = best_cl != 0;
  } else {
    c.pair_cluster = cl_saved;
    best_cl = cl_saved ? 1 : 0;
  }
  int best_eager = c.rbl_eager ? 1 : 0;
  if (c.rbl) {
    for (int v = 0; v <= 1; ++v) {
      c.rbl_eager = v != 0;
      float ms = 0.f;
      int rc = time_forces(c, reps, &ms);
      if (rc != RBE_OK) { c.timing = saved_timing; return rc; }
      if (v == 0 || ms < best) { best = ms; best_eager = v; }
    }
    c.rbl_eager = best_eager != 0;
  }
  int best_tile = c.sf_tile;
  best = 0.f;
  bool first = true;
  // the structure factor is short: several rounds of many launches, best round per tile
  const int sf_reps = std::max(20, 10 * reps);
  for (int tile = 32; tile <= 1024; tile *= 2) {
    const int64_t nblk = std::max<int64_t>(1, (c.Nq + tile - 1) / tile);
    if (nblk > c.sf_part_blocks) continue;
    set_sf_tile(c, tile);
    cudaEvent_t e0, e1;
    RBE_CUDA_TRY(cudaEventCreate(&e0));
    RBE_CUDA_TRY(cudaEventCreate(&e1));
    RBE_CUDA_TRY(launch_structure_factor(c));
    float tbest = 0.f;
    for (int round = 0; round < 3; ++round) {
      RBE_CUDA_TRY(cudaEventRecord(e0, c.stream));
      for (int r = 0; r < sf_reps; ++r) RBE_CUDA_TRY(launch_structure_factor(c));
      RBE_CUDA_TRY(cudaEventRecord(e1, c.stream));
      RBE_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (round == 0 || ms < tbest) tbest = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (first || tbest < best) { best = tbest; best_tile = tile; first = false; }
  }
  set_sf_tile(c, best_tile);
  c.timing = saved_timing;
  drop_graphs(c);
  c.have_forces = false;
  if (chosen) {
    chosen[0] = best16; chosen[1] = best_tile; chosen[2] = best_eager; chosen[3] = c.rbl_span;
    chosen[4] = best_cl;
  }
  return RBE_OK;
}

static void free_list(Ctx &c) {
  dfree(c.vl_list); dfree(c.vl_len); dfree(c.vl_listq); dfree(c.vl_lenq); dfree(c.vl_ref);
  dfree(c.s4); dfree(c.cs4); dfree(c.vl_flags); dfree(c.vl_count);
  c.vl_list = c.vl_len = c.vl_listq = c.vl_lenq = nullptr;
  c.vl_ref = nullptr;
  c.s4 = c.cs4 = nullptr;
  c.vl_flags = nullptr;
  c.vl_count = nullptr;
  c.bytes -= c.vl_bytes;
  c.vl_bytes = 0;
  c.vl_on = false;
  c.vl_skin = 0.0;
  c.vl_K = c.vl_Kq = 0;
}

// Automatic list capacity for a mean of n entries.
static int list_capacity(double n) {
  const double k = n + 6.0 * std::sqrt(n) + 32.0;
  return (int)(std::ceil(k / 8.0) * 8.0);
}

int rbe_set_neighbor_list(rbe_handle h, double skin, int capacity) {
  if (!h) return RBE_ERR_INVALID;
  Ctx &c = *h;
  if (!std::isfinite(skin) || skin < 0.0 || capacity < 0) return RBE_ERR_INVALID;
  if (c.rbl) return RBE_ERR_STATE;
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  drop_graphs(c);
  c.have_forces = false;
  free_list(c);
  if (skin == 0.0) return RBE_OK;
  const double rl = c.rc + skin;
  int R[3];
  for (int d = 0; d < 3; ++d) {
    if (!(rl < 0.5 * c.box[d])) return RBE_ERR_CUTOFF;
    const double a = c.box[d] / c.grid.n[d];
    R[d] = (int)std::ceil(rl / a);
    if (R[d] > 3 || c.grid.n[d] < 2 * R[d] + 1) return RBE_ERR_CELLS;
  }
  const double vol = c.box[0] * c.box[1] * c.box[2];
  const double sph = 4.0 / 3.0 * kPi * rl * rl * rl;
  const int K = capacity > 0 ? capacity : list_capacity((double)c.N / vol * sph);
  const int Kq = capacity > 0 ? capacity : list_capacity((double)c.Nq / vol * sph);
  const int64_t Np = (c.N + 31) / 32 * 32, Nqp = (c.Nq + 31) / 32 * 32;
  const int64_t before = c.bytes;
  int rc = RBE_OK;
  rc |= dalloc(c, &c.vl_list, Np * (int64_t)K);
  rc |= dalloc(c, &c.vl_len, c.N);
  rc |= dalloc(c, &c.vl_listq, Nqp * (int64_t)Kq);
  rc |= dalloc(c, &c.vl_lenq, c.Nq);
  rc |= dalloc(c, &c.vl_ref, 3 * c.N);
  rc |= dalloc(c, &c.s4, c.N);
  rc |= dalloc(c, &c.cs4, c.Nq);
  rc |= dalloc(c, &c.vl_flags, 8);
  rc |= dalloc(c, &c.vl_count, 2);
  c.vl_bytes = c.bytes - before;
  if (rc != RBE_OK) {
    free_list(c);
    return RBE_ERR_OOM;
  }
  RBE_CUDA_TRY(cudaMemsetAsync(c.vl_flags, 0, sizeof(int32_t) * 8, c.stream));
  RBE_CUDA_TRY(cudaMemsetAsync(c.vl_flags + 1, 1, sizeof(int32_t), c.stream));  // build first
  RBE_CUDA_TRY(cudaMemsetAsync(c.vl_count, 0, sizeof(unsigned long long) * 2, c.stream));
  RBE_CUDA_TRY(cudaMemsetAsync(c.vl_ref, 0, sizeof(uint32_t) * 3 * c.N, c.stream));
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  c.vl_on = true;
  c.vl_skin = skin;
  c.vl_K = K;
  c.vl_Kq = Kq;
  for (int d = 0; d < 3; ++d) c.vl_R[d] = R[d];
  return RBE_OK;
}

int rbe_get_neighbor_list(rbe_handle h, int64_t stats[6]) {
  if (!h || !stats) return RBE_ERR_INVALID;
  Ctx &c = *h;
  for (int k = 0; k < 6; ++k) stats[k] = 0;
  if (!c.vl_on) return RBE_OK;
  int32_t fl[8];
  unsigned long long cnt[2];
  RBE_CUDA_TRY(cudaMemcpyAsync(fl, c.vl_flags, sizeof(fl), cudaMemcpyDeviceToHost, c.stream));
  RBE_CUDA_TRY(cudaMemcpyAsync(cnt, c.vl_count, sizeof(cnt), cudaMemcpyDeviceToHost, c.stream));
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  stats[0] = (int64_t)cnt[0];
  stats[1] = (int64_t)cnt[1];
  stats[2] = fl[4];
  stats[3] = fl[5];
  stats[4] = c.vl_K;
  stats[5] = c.vl_Kq;
  return RBE_OK;
}

int rbe_get_memory(rbe_handle h, int64_t *bytes) {
  if (!h || !bytes) return RBE_ERR_INVALID;
  *bytes = h->bytes;
  return RBE_OK;
}

// A class: replicas whose Verlet steps launch the same kernels in the same shapes. Each of
// its launches runs once per step over the concatenated grids of all its replicas.
// A class: replicas whose Verlet steps launch the same kernels in the same shapes. Each of
// its kernels runs once per step over the concatenated grids of all its replicas.
struct BatchClass {
  std::vector<int> reps;
};

struct rbe_batch_s {
  std::vector<rbe_handle> h;
  std::vector<cudaStream_t> br;   // capture branches
  std::vector<cudaEvent_t> ev;    // join events
  std::vector<cudaStream_t> sub;  // per-replica launches of a class: replica r's branch
  std::vector<cudaEvent_t> sub_ev;
  std::vector<cudaEvent_t> run_ev;  // per class: fork of its per-replica launches
  cudaEvent_t fork = nullptr;
  cudaStream_t stream = nullptr;  // launch stream
  cudaStream_t cap = nullptr;     // capture origin
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  void *dev[2] = {nullptr, nullptr};  // argument tables and block prefixes of each graph
  int phase = 0;
  std::vector<int> exp_cur;       // each handle's buffer parity the graphs expect now
  bool planned = false;
  std::vector<BatchClass> cls;    // batched classes
  std::vector<int> solo;          // replicas stepped on a branch of their own
  int64_t kernels = 0;            // kernel launches per batch step
};

static void batch_drop_graphs(rbe_batch b) {
  for (int k = 0; k < 2; ++k) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    if (b->dev[k]) cudaFree(b->dev[k]);
    b->graph[k] = nullptr;
    b->dev[k] = nullptr;
  }
  b->phase = 0;
}

static int batch_free(rbe_batch b) {
  for (auto s : b->br) if (s) cudaStreamDestroy(s);
  for (auto e : b->ev) if (e) cudaEventDestroy(e);
  for (auto s : b->sub) if (s) cudaStreamDestroy(s);
  for (auto e : b->sub_ev) if (e) cudaEventDestroy(e);
  for (auto e : b->run_ev) if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  batch_drop_graphs(b);
  delete b;
  return RBE_OK;
}

// One Verlet step of replica c on c.stream (the sequence rbe_step captures).
static int step_sequence(Ctx &c) {
  if (launch_kick_drift(c) != cudaSuccess) return RBE_ERR_CUDA;  // + step counter
  int rc = force_pipeline(c, false);
  if (rc != RBE_OK) return rc;
  if (launch_kick(c) != cudaSuccess) return RBE_ERR_CUDA;
  if (c.nvt && launch_thermostat(c, 0) != cudaSuccess) return RBE_ERR_CUDA;
  if (launch_totals(c) != cudaSuccess) return RBE_ERR_CUDA;
  return RBE_OK;
}

// Record the launches of one step of replica c at buffer parity flip. Returns false when
// the step cannot run batched: a traversal without batched kernels (random batch list,
// Verlet list), a kernel without a batched form, or any other stream work, which the
// recording catches in a throwaway capture of a scratch stream.
static bool record_step(Ctx &c, int flip, Recorder &rec) {
  if (c.rbl || c.vl_on) return false;
  cudaStream_t scratch = nullptr;
  if (cudaStreamCreateWithFlags(&scratch, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int saved_cur = c.cur;
  cudaStream_t saved_stream = c.stream;
  c.cur = flip ? 1 - saved_cur : saved_cur;
  c.stream = scratch;
  c.rec = &rec;
  bool ok = cudaStreamBeginCapture(scratch, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    ok = step_sequence(c) == RBE_OK && rec.ok;
    cudaGraph_t g = nullptr;
    size_t nodes = 0;
    if (cudaStreamEndCapture(scratch, &g) != cudaSuccess) ok = false;
    if (g) {
      if (cudaGraphGetNodes(g, nullptr, &nodes) != cudaSuccess || nodes != 0) ok = false;
      cudaGraphDestroy(g);
    }
  }
  c.rec = nullptr;
  c.cur = saved_cur;
  c.stream = saved_stream;
  cudaStreamDestroy(scratch);
  cudaGetLastError();
  return ok;
}

// Same kernel (batched and solo: a kernel launched per replica has no batched form, so its
// solo instance decides) and the same block shape.
static bool same_shape(const RecItem &x, const RecItem &y) {
  return x.fn == y.fn && x.solo_fn == y.solo_fn && x.per_replica == y.per_replica &&
         x.grid.y == y.grid.y && x.grid.z == y.grid.z &&
         x.block.x == y.block.x && x.block.y == y.block.y && x.block.z == y.block.z &&
         x.smem == y.smem && x.args.size() == y.args.size();
}
static bool same_sequence(const Recorder &x, const Recorder &y) {
  if (x.items.size() != y.items.size()) return false;
  for (size_t i = 0; i < x.items.size(); ++i)
    if (!same_shape(x.items[i], y.items[i])) return false;
  return true;
}

// Group the replicas into classes by the kernels and shapes of their steps (at both
// buffer parities); a class of one gains nothing and steps on its own branch.
static int batch_plan(rbe_batch b) {
  const int n = (int)b->h.size();
  std::vector<Recorder> rec(n);
  std::vector<bool> ok(n);
  for (int r = 0; r < n; ++r) {
    Recorder other;
    ok[r] = record_step(*b->h[r], 0, rec[r]) && record_step(*b->h[r], 1, other) &&
            same_sequence(rec[r], other);
  }
  b->cls.clear();
  b->solo.clear();
  for (int r = 0; r < n; ++r) {
    if (!ok[r]) {
      b->solo.push_back(r);
      continue;
    }
    bool placed = false;
    for (auto &k : b->cls)
      if (same_sequence(rec[k.reps[0]], rec[r])) {
        k.reps.push_back(r);
        placed = true;
        break;
      }
    if (!placed) b->cls.push_back(BatchClass{{r}});
  }
  for (size_t k = 0; k < b->cls.size();) {
    if (b->cls[k].reps.size() < 2) {
      b->solo.push_back(b->cls[k].reps[0]);
      b->cls.erase(b->cls.begin() + k);
    } else {
      ++k;
    }
  }
  std::sort(b->solo.begin(), b->solo.end());
  b->kernels = 0;
  for (auto &k : b->cls)
    for (size_t i = 0; i < rec[k.reps[0]].items.size(); ++i) {
      int64_t blocks = 0, launches = 0;
      for (int r : k.reps) {
        blocks += rec[r].items[i].grid.x;
        launches += rec[r].items[i].grid.x > 0 ? 1 : 0;
      }
      if (rec[k.reps[0]].items[i].per_replica) b->kernels += launches;
      else if (blocks > 0) b->kernels += 1;
    }
  for (int r : b->solo) b->kernels += kernels_per_step(*b->h[r]);
  b->planned = true;
  return RBE_OK;
}

// One launch of a class: the batched kernel, the concatenated grid, and its tables; or,
// for a kernel launched per replica, the solo kernel with each replica's grid and arguments.
struct ClassLaunch {
  const void *fn;
  dim3 grid, block;
  size_t smem, tab_off, pre_off;
  bool per_replica;
  std::vector<dim3> grids;
  std::vector<std::vector<unsigned char>> args;
};

// Record every class's step at buffer parity flip, lay the argument tables and block
// prefixes out in one device buffer (uploaded here) and return the launches.
static int batch_tables(rbe_batch b, int flip, void **dev, std::vector<std::vector<ClassLaunch>> &out) {
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  std::vector<std::vector<Recorder>> rec(b->cls.size());
  size_t bytes = 0;
  out.assign(b->cls.size(), {});
  for (size_t k = 0; k < b->cls.size(); ++k) {
    const auto &reps = b->cls[k].reps;
    rec[k].resize(reps.size());
    for (size_t j = 0; j < reps.size(); ++j)
      if (!record_step(*b->h[reps[j]], flip, rec[k][j]) || !same_sequence(rec[k][0], rec[k][j]))
        return RBE_ERR_STATE;  // a handle's configuration changed since the plan
    for (size_t i = 0; i < rec[k][0].items.size(); ++i) {
      const RecItem &it = rec[k][0].items[i];
      ClassLaunch L;
      L.block = it.block;
      L.smem = it.smem;
      L.per_replica = it.per_replica;
      L.tab_off = L.pre_off = 0;
      if (it.per_replica) {
        L.fn = it.solo_fn;
        L.grid = it.grid;
        for (size_t j = 0; j < reps.size(); ++j) {
          L.grids.push_back(rec[k][j].items[i].grid);
          L.args.push_back(rec[k][j].items[i].args);
        }
      } else {
        L.fn = it.fn;
        L.grid = dim3(0, it.grid.y, it.grid.z);
        L.tab_off = bytes;
        bytes = align(bytes + it.args.size() * reps.size());
        L.pre_off = bytes;
        bytes = align(bytes + sizeof(int32_t) * (reps.size() + 1));
      }
      out[k].push_back(std::move(L));
    }
  }
  std::vector<unsigned char> host(bytes, 0);
  for (size_t k = 0; k < b->cls.size(); ++k)
    for (size_t i = 0; i < out[k].size(); ++i) {
      ClassLaunch &L = out[k][i];
      if (L.per_replica) continue;
      const size_t sz = rec[k][0].items[i].args.size();
      int32_t *pp = reinterpret_cast<int32_t *>(host.data() + L.pre_off);
      int64_t pre = 0;
      for (size_t j = 0; j < rec[k].size(); ++j) {
        const RecItem &it = rec[k][j].items[i];
        std::memcpy(host.data() + L.tab_off + j * sz, it.args.data(), sz);
        pp[j] = (int32_t)pre;
        pre += it.grid.x;
        if (pre > INT32_MAX) return RBE_ERR_INVALID;
      }
      pp[rec[k].size()] = (int32_t)pre;
      L.grid.x = (unsigned)pre;
    }
  *dev = nullptr;
  if (bytes == 0) return RBE_OK;
  if (cudaMalloc(dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    *dev = nullptr;
    return RBE_ERR_OOM;
  }
  RBE_CUDA_TRY(cudaMemcpy(*dev, host.data(), bytes, cudaMemcpyHostToDevice));
  return RBE_OK;
}

// Graph k: fork from the origin stream; each class's launches in order on a branch of its
// own, and each remaining replica's Verlet step on a branch of its own; join. `flip`
// selects the buffer parity relative to the handles' current one.
static int batch_capture(rbe_batch b, int k, int flip) {
  const int n = (int)b->h.size();
  std::vector<std::vector<ClassLaunch>> launches;
  int rc = batch_tables(b, flip, &b->dev[k], launches);
  if (rc != RBE_OK) return rc;
  std::vector<int> saved_cur(n);
  std::vector<cudaStream_t> saved_stream(n);
  for (int r = 0; r < n; ++r) {
    saved_cur[r] = b->h[r]->cur;
    saved_stream[r] = b->h[r]->stream;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaEventRecord(b->fork, b->cap);
    int nb = 0;  // branches used
    for (size_t kc = 0; kc < b->cls.size() && rc == RBE_OK; ++kc) {
      cudaStream_t st = b->br[nb];
      if (cudaStreamWaitEvent(st, b->fork, 0) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
      const auto &reps = b->cls[kc].reps;
      int nrep = (int)reps.size();
      const auto &Ls = launches[kc];
      for (size_t i = 0; i < Ls.size() && rc == RBE_OK;) {
        if (Ls[i].per_replica) {
          // a run of per-replica launches: fork one branch per replica, then join
          size_t i1 = i;
          while (i1 < Ls.size() && Ls[i1].per_replica) ++i1;
          if (cudaEventRecord(b->run_ev[kc], st) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
          for (int j = 0; j < nrep && rc == RBE_OK; ++j) {
            cudaStream_t ss = b->sub[reps[j]];
            if (cudaStreamWaitEvent(ss, b->run_ev[kc], 0) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
            for (size_t q = i; q < i1; ++q) {
              const ClassLaunch &L = Ls[q];
              const dim3 g = L.grids[j];
              if (g.x == 0) continue;
              void *params[] = {const_cast<unsigned char *>(L.args[j].data())};
              if (cudaLaunchKernel(L.fn, g, L.block, params, L.smem, ss) != cudaSuccess) {
                rc = RBE_ERR_CUDA;
                break;
              }
            }
            if (rc != RBE_OK) break;
            cudaEventRecord(b->sub_ev[reps[j]], ss);
            cudaStreamWaitEvent(st, b->sub_ev[reps[j]], 0);
          }
          i = i1;
          continue;
        }
        const ClassLaunch &L = Ls[i++];
        if (L.grid.x == 0) continue;
        const void *tab = static_cast<char *>(b->dev[k]) + L.tab_off;
        const void *pre = static_cast<char *>(b->dev[k]) + L.pre_off;
        void *params[] = {&tab, &pre, &nrep};
        if (cudaLaunchKernel(L.fn, L.grid, L.block, params, L.smem, st) != cudaSuccess) {
          rc = RBE_ERR_CUDA;
          break;
        }
      }
      if (rc != RBE_OK) break;
      cudaEventRecord(b->ev[nb], st);
      cudaStreamWaitEvent(b->cap, b->ev[nb], 0);
      ++nb;
    }
    for (size_t j = 0; j < b->solo.size() && rc == RBE_OK; ++j) {
      Ctx &c = *b->h[b->solo[j]];
      cudaStream_t st = b->br[nb];
      c.cur = flip ? 1 - c.cur : c.cur;
      c.stream = st;
      if (cudaStreamWaitEvent(st, b->fork, 0) != cudaSuccess) { rc = RBE_ERR_CUDA; break; }
      rc = step_sequence(c);
      if (rc != RBE_OK) break;
      cudaEventRecord(b->ev[nb], st);
      cudaStreamWaitEvent(b->cap, b->ev[nb], 0);
      ++nb;
    }
    e = cudaStreamEndCapture(b->cap, &g);
  }
  for (int r = 0; r < n; ++r) {
    b->h[r]->cur = saved_cur[r];
    b->h[r]->stream = saved_stream[r];
  }
  if (rc != RBE_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  RBE_CUDA_TRY(e);
  e = cudaGraphInstantiate(&b->graph[k], g, 0);
  cudaGraphDestroy(g);
  RBE_CUDA_TRY(e);
  return RBE_OK;
}

int rbe_batch_create(rbe_batch *out, int n, const rbe_handle *handles, void *cuda_stream) {
  if (!out || n < 1 || !handles) return RBE_ERR_INVALID;
  *out = nullptr;
  for (int r = 0; r < n; ++r)
    if (!handles[r]) return RBE_ERR_INVALID;
  rbe_batch b = new (std::nothrow) rbe_batch_s();
  if (!b) return RBE_ERR_OOM;
  b->h.assign(handles, handles + n);
  b->stream = (cudaStream_t)cuda_stream;
  b->br.assign(n, nullptr);
  b->ev.assign(n, nullptr);
  b->sub.assign(n, nullptr);
  b->sub_ev.assign(n, nullptr);
  b->run_ev.assign(n, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int r = 0; r < n && ok; ++r)
    ok = cudaStreamCreateWithFlags(&b->br[r], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev[r], cudaEventDisableTiming) == cudaSuccess &&
         cudaStreamCreateWithFlags(&b->sub[r], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->sub_ev[r], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->run_ev[r], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    batch_free(b);
    return RBE_ERR_CUDA;
  }
  *out = b;
  return RBE_OK;
}

int rbe_batch_step(rbe_batch b, int nsteps) {
  if (!b || nsteps < 0) return RBE_ERR_INVALID;
  if (nsteps == 0) return RBE_OK;
  // initial forces (and thermostat start halves) of every replica on its own stream, then
  // order the batch stream after them
  for (auto h : b->h) {
    if (!h->have_forces) {
      int rc = forces_common(h, h->step, false);
      if (rc != RBE_OK) return rc;
    }
    if (h->nvt && !h->nvt_primed) {
      RBE_CUDA_TRY(launch_kinetic(*h));
      RBE_CUDA_TRY(launch_thermostat(*h, 1));
      h->nvt_primed = true;
    }
    RBE_CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  if (!b->planned) {
    const int rc = batch_plan(b);
    if (rc != RBE_OK) return rc;
  }
  // the graphs hold buffer pointers by parity: capture them again when a handle's parity is
  // not the one they expect (the handle stepped on its own in between)
  bool moved = b->exp_cur.size() != b->h.size();
  for (size_t r = 0; r < b->exp_cur.size() && !moved; ++r) moved = b->exp_cur[r] != b->h[r]->cur;
  if (moved) {
    batch_drop_graphs(b);
    b->exp_cur.resize(b->h.size());
    for (size_t r = 0; r < b->h.size(); ++r) b->exp_cur[r] = b->h[r]->cur;
  }
  for (int k = 0; k < 2; ++k)
    if (!b->graph[k]) {
      // graph k serves the steps at phase k: parity (phase + k) relative to now
      const int rc = batch_capture(b, k, (b->phase + k) & 1);
      if (rc != RBE_OK) {
        batch_drop_graphs(b);
        b->exp_cur.clear();
        return rc;
      }
    }
  for (int s = 0; s < nsteps; ++s) {
    RBE_CUDA_TRY(cudaGraphLaunch(b->graph[b->phase], b->stream));
    b->phase ^= 1;
    for (size_t r = 0; r < b->h.size(); ++r) {
      rbe_handle h = b->h[r];
      h->cur = 1 - h->cur;
      h->step += 1;
      h->have_forces = true;
      b->exp_cur[r] = h->cur;
    }
  }
  return RBE_OK;
}

int rbe_batch_info(rbe_batch b, int32_t *n_classes, int32_t *n_batched, int64_t *kernels) {
  if (!b) return RBE_ERR_INVALID;
  if (!b->planned) {
    const int rc = batch_plan(b);
    if (rc != RBE_OK) return rc;
  }
  int32_t nb = 0;
  for (auto &k : b->cls) nb += (int32_t)k.reps.size();
  if (n_classes) *n_classes = (int32_t)b->cls.size();
  if (n_batched) *n_batched = nb;
  if (kernels) *kernels = b->kernels;
  return RBE_OK;
}

int rbe_batch_destroy(rbe_batch b) {
  if (!b) return RBE_OK;
  cudaStreamSynchronize(b->stream);
  return batch_free(b);
}

// ---------------------------------------------------------------------------------------
// Checkpoint / resume. File layout (little-endian, native sizes):
//   "RBECKPT1"; the fingerprint (N, box, alpha, r_c, r_core, C, dt, kappa, P, p_rbl,
//   precision, n_types, seed, replica, the LJ A/B table); the step counter; the thermostat
//   (on, T, tau, kB, primed, its 7 device scalars); s (N x 3 uint32) and v (N x 3 double), id
//   order.
namespace {
const char kCkptMagic[8] = {'R', 'B', 'E', 'C', 'K', 'P', 'T', '1'};

struct CkptHead {
  int64_t N;
  double box[3], alpha, rc, r_core, C, dt, kappa;
  int32_t P, p_rbl, precision, nt;
  uint64_t seed;
  uint32_t replica, pad;
  double ljA[kMaxTypes * kMaxTypes], ljB[kMaxTypes * kMaxTypes];
  uint64_t step;
  int32_t nvt, primed;
  double T0, tau, kB, thermo[7];
};

void ckpt_head(const Ctx &c, CkptHead &hd) {
  std::memset(&hd, 0, sizeof(hd));
  hd.N = c.N;
  for (int d = 0; d < 3; ++d) hd.box[d] = c.box[d];
  hd.alpha = c.alpha; hd.rc = c.rc; hd.r_core = c.r_core; hd.C = c.C; hd.dt = c.dt;
  hd.kappa = c.kappa; hd.P = c.P; hd.p_rbl = c.p_rbl; hd.precision = c.precision; hd.nt = c.nt;
  hd.seed = c.seed; hd.replica = c.replica;
  for (int k = 0; k < c.nt * c.nt; ++k) { hd.ljA[k] = c.lj.Ad[k]; hd.ljB[k] = c.lj.Bd[k]; }
}
}  // namespace

int rbe_save(rbe_handle h, const char *path) {
  if (!h || !path) return RBE_ERR_INVALID;
  Ctx &c = *h;
  CkptHead hd;
  ckpt_head(c, hd);
  hd.step = c.step;
  hd.nvt = c.nvt ? 1 : 0;
  hd.primed = c.nvt_primed ? 1 : 0;
  hd.T0 = c.T0; hd.tau = c.tau; hd.kB = c.kB;
  if (c.thermo) {
    RBE_CUDA_TRY(cudaMemcpyAsync(hd.thermo, c.thermo, sizeof(hd.thermo), cudaMemcpyDeviceToHost,
                                 c.stream));
  }
  std::vector<uint32_t> s(3 * (size_t)c.N);
  std::vector<double> v(3 * (size_t)c.N);
  int rc = rbe_get_state(h, nullptr, v.data(), s.data());  // synchronises
  if (rc != RBE_OK) return rc;
  FILE *f = std::fopen(path, "wb");
  if (!f) return RBE_ERR_INVALID;
  bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
            std::fwrite(s.data(), sizeof(uint32_t), s.size(), f) == s.size() &&
            std::fwrite(v.data(), sizeof(double), v.size(), f) == v.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? RBE_OK : RBE_ERR_INVALID;
}

int rbe_load(rbe_handle h, const char *path) {
  if (!h || !path) return RBE_ERR_INVALID;
  Ctx &c = *h;
  FILE *f = std::fopen(path, "rb");
  if (!f) return RBE_ERR_INVALID;
  char magic[8];
  CkptHead hd;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
            std::fread(&hd, sizeof(hd), 1, f) == 1;
  if (!ok) { std::fclose(f); return RBE_ERR_INVALID; }
  CkptHead mine;
  ckpt_head(c, mine);
  // the checkpoint must come from a handle with the same system and parameters
  const size_t fp = offsetof(CkptHead, step);
  if (std::memcmp(&hd, &mine, fp) != 0) { std::fclose(f); return RBE_ERR_STATE; }
  std::vector<uint32_t> s(3 * (size_t)c.N);
  std::vector<double> v(3 * (size_t)c.N);
  ok = std::fread(s.data(), sizeof(uint32_t), s.size(), f) == s.size() &&
       std::fread(v.data(), sizeof(double), v.size(), f) == v.size();
  std::fclose(f);
  if (!ok) return RBE_ERR_INVALID;
  for (double x : v)
    if (!std::isfinite(x)) return RBE_ERR_INVALID;
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  // staging: the positions in the 3N-float buffer, the velocities in the 3N-double one
  RBE_CUDA_TRY(cudaMemcpy(c.outf, s.data(), sizeof(uint32_t) * s.size(), cudaMemcpyHostToDevice));
  RBE_CUDA_TRY(cudaMemcpy(c.pos_stage, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice));
  RBE_CUDA_TRY(launch_gather_state(c, reinterpret_cast<const uint32_t *>(c.outf), c.pos_stage));
  c.step = hd.step;
  RBE_CUDA_TRY(launch_set_step(c, c.step));
  if (hd.nvt) {
    int rs = rbe_set_thermostat(h, hd.T0, hd.tau, hd.kB);
    if (rs != RBE_OK) return rs;
    RBE_CUDA_TRY(cudaMemcpy(c.thermo, hd.thermo, sizeof(hd.thermo), cudaMemcpyHostToDevice));
    c.nvt_primed = hd.primed != 0;
  } else if (c.nvt) {
    int rs = rbe_set_thermostat(h, 0.0, 0.0, 0.0);
    if (rs != RBE_OK) return rs;
  }
  drop_graphs(c);
  c.have_forces = false;  // the next step evaluates the forces of the loaded state
  RBE_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return RBE_OK;
}

int rbe_check_device(rbe_handle h) {
  if (!h) return RBE_ERR_INVALID;
  return read_device_flags(*h);
}

}  // extern "C"
