// k_integrate.cu -- velocity Verlet on the fixed-point grid, energy totals, and the
// gathers that translate between cell-sorted storage and caller id order.
//
// Velocity Verlet (the time integrator of Sec. 2.1):
//   v += (F/m)(dt/2) kappa;  s += rint(v dt 2^32 / L)  (FP64 increment, wraps mod 2^32)
//   ... forces at the new positions ...;  v += (F/m)(dt/2) kappa
// Every kernel here is a single streaming pass (HBM-bound) except the totals, which sum
// the per-block partials of all force kernels in a fixed order (latency-bound).
#include "rbe_internal.cuh"

namespace rbe {

int64_t rbl_compact_count(int64_t nblk);

// g_d = dt 2^32 / L_d (FP64, from the host): the fixed-point increment is rint(v g_d), in
// FP64 in the FP64 form. The FP32 forms round the FP32 product (off by at most one grid unit
// of L / 2^32 where the FP64 rounding would differ); FP64 runs at 1/64 of the FP32 rate on
// this GPU, and this pass would otherwise be bound by it instead of by memory.
template <typename V, typename FT>
__global__ void kick_drift_kernel(V *__restrict__ v, const FT *__restrict__ F,
                                  const float *__restrict__ invm, uint32_t *__restrict__ s,
                                  int64_t N, double hdk, double gx, double gy, double gz,
                                  int *__restrict__ err, const double *__restrict__ scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double g[3] = {gx, gy, gz};
  const V im = (V)invm[i];
  const V sc = scale ? (V)*scale : (V)1;  // Nose-Hoover start-of-step scaling
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    V vv = v[d * N + i] * sc + (V)F[d * N + i] * im * (V)hdk;
    v[d * N + i] = vv;
    int st;
    if (sizeof(V) == 8) {
      const double inc = (double)vv * g[d];
      bad |= !isfinite(inc) || fabs(inc) > 2.0e9;
      st = bad ? 0 : __double2int_rn(inc);
    } else {
      const float inc = (float)vv * (float)g[d];
      bad |= !isfinite(inc) || fabsf(inc) > 2.0e9f;
      st = bad ? 0 : __float2int_rn(inc);
    }
    s[d * N + i] += (uint32_t)st;
  }
  if (bad) atomicOr(err, ERRBIT_NONFINITE);
}

template <typename V, typename FT>
__global__ void __launch_bounds__(256)
    kick_kernel(V *__restrict__ v, const FT *__restrict__ F, const float *__restrict__ invm,
                int64_t N, double hdk, double inv_kappa, int do_kick,
                double *__restrict__ ke_part) {
  __shared__ double sh[256];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double ke = 0.0;
  if (i < N) {
    const V im = (V)invm[i];
    V v2 = (V)0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      V vv = v[d * N + i];
      if (do_kick) {
        vv += (V)F[d * N + i] * im * (V)hdk;
        v[d * N + i] = vv;
      }
      v2 += vv * vv;
    }
    // 1/2 m v^2 / kappa, m = 1 / (1/m): FP64 in the FP64 form; the FP32 forms form each
    // particle's term in FP32 and sum the terms in FP64
    if (sizeof(V) == 8) ke = 0.5 * (double)v2 / (double)invm[i] * inv_kappa;
    else ke = (double)(0.5f * (float)v2 * __frcp_rn(invm[i]) * (float)inv_kappa);
  }
  sh[threadIdx.x] = ke;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) ke_part[blockIdx.x] = sh[0];
}

// Nose-Hoover half steps (chain of one): from 2K = 2 sum(kinetic partials) the end-of-step
// half (mode 0) gives the velocity scale s_end and the start-of-next-step half gives
// s_start, applied by the next kick-drift; mode 1 only does the start half (first step).
__global__ void __launch_bounds__(256)
    thermostat_kernel(const double *__restrict__ ke_part, int64_t n, double Nf, double kT,
                      double Q, double dt, double *__restrict__ th, int mode) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t b = threadIdx.x; b < n; b += blockDim.x) acc += ke_part[b];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double K2 = 2.0 * sh[0];
  double xi = th[0], eta = th[1], s_end = 1.0;
  if (mode == 0) {
    xi += 0.25 * dt * (K2 - Nf * kT) / Q;
    s_end = exp(-xi * 0.5 * dt);
    K2 *= s_end * s_end;
    eta += xi * 0.5 * dt;
    xi += 0.25 * dt * (K2 - Nf * kT) / Q;
  }
  th[3] = 0.5 * K2;
  th[4] = s_end;
  th[5] = xi;   // state at the end of the step (reported)
  th[6] = eta;
  xi += 0.25 * dt * (K2 - Nf * kT) / Q;
  const double s_start = exp(-xi * 0.5 * dt);
  K2 *= s_start * s_start;
  eta += xi * 0.5 * dt;
  xi += 0.25 * dt * (K2 - Nf * kT) / Q;
  th[0] = xi;
  th[1] = eta;
  th[2] = s_start;
}

template <typename V>
__global__ void scale_v_kernel(V *__restrict__ v, int64_t N, const double *__restrict__ scale) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 3 * N) return;
  v[k] *= (V)*scale;
}

struct TotalsArgs {
  const double *ke_override;
  const double *pair, *coul, *rbl, *ke, *emode;
  int64_t n_pair, n_coul, n_rbl, n_ke;
  int P;
  double U_self;
  double *scal;
};

// Fixed-order reduction of every partial into the scalars (ACC = float for the plain
// FP32 form, double otherwise). One block of kTotalsThreads: strided per-thread sums (four
// partials in flight per thread), then warp shuffles, then the warp sums in order.
constexpr int kTotalsThreads = 1024;

template <typename ACC>
__global__ void __launch_bounds__(kTotalsThreads) totals_kernel(TotalsArgs a) {
  constexpr int NV = 7;  // ureal ulj wreal wlj uk wk ke
  constexpr int NW = kTotalsThreads / 32;
  __shared__ ACC sh[NV][NW];
  ACC acc[NV];
  for (int k = 0; k < NV; ++k) acc[k] = (ACC)0;
  const double *srcs[3] = {a.pair, a.coul, a.rbl};
  const int64_t ns[3] = {a.n_pair, a.n_coul, a.n_rbl};
  for (int r = 0; r < 3; ++r) {
#pragma unroll 4
    for (int64_t b = threadIdx.x; b < ns[r]; b += blockDim.x)
      for (int k = 0; k < NQ_PAIR; ++k) acc[k] += (ACC)srcs[r][b * NQ_PAIR + k];
  }
  for (int l = threadIdx.x; l < a.P; l += blockDim.x) {
    acc[4] += (ACC)a.emode[2 * l];
    acc[5] += (ACC)a.emode[2 * l + 1];
  }
  for (int64_t b = threadIdx.x; b < a.n_ke; b += blockDim.x) acc[6] += (ACC)a.ke[b];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < NV; ++k) {
    const ACC v = warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    ACC t = (ACC)0;
    for (int w = 0; w < NW; ++w) t += sh[threadIdx.x][w];
    sh[threadIdx.x][0] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double ur = (double)sh[Q_UREAL][0], ul = (double)sh[Q_ULJ][0];
    const double wr = (double)sh[Q_WREAL][0], wl = (double)sh[Q_WLJ][0];
    const double uk = (double)sh[4][0], wk = (double)sh[5][0];
    const double ke = a.ke_override ? *a.ke_override : (double)sh[6][0];
    a.scal[S_UREAL] = ur;
    a.scal[S_ULJ] = ul;
    a.scal[S_UK] = uk;
    a.scal[S_USELF] = a.U_self;
    a.scal[S_UTOT] = ur + ul + uk - a.U_self;
    a.scal[S_KE] = ke;
    a.scal[S_WREAL] = wr;
    a.scal[S_WLJ] = wl;
    a.scal[S_WK] = wk;
    a.scal[S_WTOT] = wr + wl + wk;
  }
}

template <typename FT, typename OT>
__global__ void scatter_forces_kernel(const FT *__restrict__ F, const int32_t *__restrict__ id,
                                      int64_t N, OT *__restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t o = (int64_t)id[k] * 3;
  out[o] = (OT)F[k];
  out[o + 1] = (OT)F[N + k];
  out[o + 2] = (OT)F[2 * N + k];
}

template <typename V>
__global__ void scatter_state_kernel(const uint32_t *__restrict__ s, const V *__restrict__ v,
                                     const int32_t *__restrict__ id, int64_t N, int what,
                                     double hx, double hy, double hz, double *__restrict__ outd,
                                     uint32_t *__restrict__ outu) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t o = (int64_t)id[k] * 3;
  if (what == 0) {
    outd[o] = (double)s[k] * hx;
    outd[o + 1] = (double)s[N + k] * hy;
    outd[o + 2] = (double)s[2 * N + k] * hz;
  } else if (what == 1) {
    outd[o] = (double)v[k];
    outd[o + 1] = (double)v[N + k];
    outd[o + 2] = (double)v[2 * N + k];
  } else {
    outu[o] = s[k];
    outu[o + 1] = s[N + k];
    outu[o + 2] = s[2 * N + k];
  }
}

__global__ void set_positions_kernel(const double *__restrict__ pos, const int32_t *__restrict__ id,
                                     int64_t N, double Lx, double Ly, double Lz,
                                     uint32_t *__restrict__ s) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t o = (int64_t)id[k] * 3;
  const double L[3] = {Lx, Ly, Lz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double f = __dmul_rn(__ddiv_rn(pos[o + d], L[d]), kTwo32);
    const double fm = f - kTwo32 * floor(f / kTwo32);  // wrap into [0, 2^32)
    s[d * N + k] = (uint32_t)(unsigned long long)__double2ll_rn(fm);
  }
}

// Checkpoint load: state given in id order (row-major per particle) into the sorted slots.
template <typename V>
__global__ void gather_state_kernel(const uint32_t *__restrict__ s_id, const double *__restrict__ v_id,
                                    const int32_t *__restrict__ id, int64_t N,
                                    uint32_t *__restrict__ s, V *__restrict__ v) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t o = (int64_t)id[k] * 3;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    s[d * N + k] = s_id[o + d];
    v[d * N + k] = (V)v_id[o + d];
  }
}

__global__ void scatter_int_kernel(const int32_t *__restrict__ src, const int32_t *__restrict__ id,
                                   int64_t N, int width, int32_t *__restrict__ dst) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t o = (int64_t)id[k] * width;
  for (int w = 0; w < width; ++w) dst[o + w] = src[k * width + w];
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_kick_drift(Ctx &c) {
  const int b = c.cur;
  const double hdk = 0.5 * c.dt * c.kappa;
  if (c.N == 0) return cudaSuccess;
  const double *scale = c.nvt ? c.thermo + 2 : nullptr;
  const double gx = c.dt * kTwo32 / c.box[0], gy = c.dt * kTwo32 / c.box[1],
               gz = c.dt * kTwo32 / c.box[2];
  if (c.precision == RBE_FP64)
    kick_drift_kernel<double, double><<<nblk(c.N, 256), 256, 0, c.stream>>>(
        c.vd[b], c.Fd, c.invm[b], c.s[b], c.N, hdk, gx, gy, gz, c.err, scale);
  else
    kick_drift_kernel<float, float><<<nblk(c.N, 256), 256, 0, c.stream>>>(
        c.vf[b], c.F, c.invm[b], c.s[b], c.N, hdk, gx, gy, gz, c.err, scale);
  return cudaGetLastError();
}

cudaError_t launch_thermostat(Ctx &c, int mode) {
  const int b = c.cur;
  thermostat_kernel<<<1, 256, 0, c.stream>>>(c.epart + c.off_ke, c.n_ke_blk, c.Nf, c.kB * c.T0,
                                             c.Qnh, c.dt, c.thermo, mode);
  if (mode == 0) {
    if (c.precision == RBE_FP64)
      scale_v_kernel<double><<<nblk(3 * c.N, 256), 256, 0, c.stream>>>(c.vd[b], c.N, c.thermo + 4);
    else
      scale_v_kernel<float><<<nblk(3 * c.N, 256), 256, 0, c.stream>>>(c.vf[b], c.N, c.thermo + 4);
  }
  return cudaGetLastError();
}

static cudaError_t kick_impl(Ctx &c, int do_kick) {
  const int b = c.cur;
  const double hdk = 0.5 * c.dt * c.kappa;
  if (c.N == 0) return cudaSuccess;
  if (c.precision == RBE_FP64)
    kick_kernel<double, double><<<nblk(c.N, 256), 256, 0, c.stream>>>(
        c.vd[b], c.Fd, c.invm[b], c.N, hdk, 1.0 / c.kappa, do_kick, c.epart + c.off_ke);
  else
    kick_kernel<float, float><<<nblk(c.N, 256), 256, 0, c.stream>>>(
        c.vf[b], c.F, c.invm[b], c.N, hdk, 1.0 / c.kappa, do_kick, c.epart + c.off_ke);
  return cudaGetLastError();
}

cudaError_t launch_kick(Ctx &c) { return kick_impl(c, 1); }
cudaError_t launch_kinetic(Ctx &c) { return kick_impl(c, 0); }

// Block partials of a pair pass ([nblk][NQ_PAIR]) summed over fixed contiguous ranges in a
// fixed order into [gridDim.x][NQ_PAIR]: the FP64 adds are spread over many SMs (one SM's
// FP64 rate is low) before the one-block totals.
__global__ void __launch_bounds__(256) partials_compact_kernel(const double *__restrict__ in,
                                                               int64_t nblk, int64_t per,
                                                               double *__restrict__ out) {
  __shared__ double sh[NQ_PAIR][256];
  const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(nblk, b0 + per);
  double acc[NQ_PAIR];
#pragma unroll
  for (int k = 0; k < NQ_PAIR; ++k) acc[k] = 0.0;
  for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NQ_PAIR; ++k) acc[k] += in[b * NQ_PAIR + k];
#pragma unroll
  for (int k = 0; k < NQ_PAIR; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st)
#pragma unroll
      for (int k = 0; k < NQ_PAIR; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < NQ_PAIR) out[(int64_t)blockIdx.x * NQ_PAIR + threadIdx.x] = sh[threadIdx.x][0];
}

int64_t partials_compact_count(int64_t nblk) { return std::min<int64_t>(nblk, kCompactMax); }

cudaError_t launch_totals(Ctx &c) {
  TotalsArgs a;
  // pair and Coulomb-pass partials, compacted first (at most kCompactMax per pass)
  const int64_t ncp = partials_compact_count(c.n_pair_blk), ncc = partials_compact_count(c.n_coul_blk);
  if (ncp > 0)
    partials_compact_kernel<<<(unsigned)ncp, 256, 0, c.stream>>>(
        c.epart + c.off_pair, c.n_pair_blk, (c.n_pair_blk + ncp - 1) / ncp, c.ecomp);
  if (ncc > 0)
    partials_compact_kernel<<<(unsigned)ncc, 256, 0, c.stream>>>(
        c.epart + c.off_coul, c.n_coul_blk, (c.n_coul_blk + ncc - 1) / ncc,
        c.ecomp + kCompactMax * NQ_PAIR);
  a.pair = c.ecomp; a.n_pair = ncp;
  a.coul = c.ecomp + kCompactMax * NQ_PAIR; a.n_coul = ncc;
  // RBL partials: the compacted ones (rbl_compact_kernel runs after the RBL kernel)
  a.rbl = c.rbl ? c.rbl_cpart : c.epart + c.off_rbl;
  a.n_rbl = c.rbl ? rbl_compact_count(c.n_rbl_blk) : 0;
  a.ke = c.epart + c.off_ke; a.n_ke = c.n_ke_blk;
  a.emode = c.emode; a.P = c.P;
  a.U_self = c.U_self;
  a.scal = c.scal;
  a.ke_override = c.nvt ? c.thermo + 3 : nullptr;
  if (c.precision == RBE_FP32) totals_kernel<float><<<1, kTotalsThreads, 0, c.stream>>>(a);
  else totals_kernel<double><<<1, kTotalsThreads, 0, c.stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scatter_forces(Ctx &c, bool to_double) {
  const int b = c.cur;
  if (c.N == 0) return cudaSuccess;
  if (c.precision == RBE_FP64) {
    if (to_double) scatter_forces_kernel<double, double><<<nblk(c.N, 256), 256, 0, c.stream>>>(c.Fd, c.id[b], c.N, c.outd);
    else scatter_forces_kernel<double, float><<<nblk(c.N, 256), 256, 0, c.stream>>>(c.Fd, c.id[b], c.N, c.outf);
  } else {
    if (to_double) scatter_forces_kernel<float, double><<<nblk(c.N, 256), 256, 0, c.stream>>>(c.F, c.id[b], c.N, c.outd);
    else scatter_forces_kernel<float, float><<<nblk(c.N, 256), 256, 0, c.stream>>>(c.F, c.id[b], c.N, c.outf);
  }
  return cudaGetLastError();
}

cudaError_t launch_scatter_state(Ctx &c, int what) {
  const int b = c.cur;
  if (c.N == 0) return cudaSuccess;
  const double hx = c.box[0] / kTwo32, hy = c.box[1] / kTwo32, hz = c.box[2] / kTwo32;
  uint32_t *outu = reinterpret_cast<uint32_t *>(c.outf);
  if (c.precision == RBE_FP64)
    scatter_state_kernel<double><<<nblk(c.N, 256), 256, 0, c.stream>>>(c.s[b], c.vd[b], c.id[b], c.N, what, hx, hy, hz, c.outd, outu);
  else
    scatter_state_kernel<float><<<nblk(c.N, 256), 256, 0, c.stream>>>(c.s[b], c.vf[b], c.id[b], c.N, what, hx, hy, hz, c.outd, outu);
  return cudaGetLastError();
}

cudaError_t launch_set_positions(Ctx &c) {
  const int b = c.cur;
  if (c.N == 0) return cudaSuccess;
  set_positions_kernel<<<nblk(c.N, 256), 256, 0, c.stream>>>(c.pos_stage, c.id[b], c.N, c.box[0],
                                                             c.box[1], c.box[2], c.s[b]);
  return cudaGetLastError();
}

cudaError_t launch_gather_state(Ctx &c, const uint32_t *s_id, const double *v_id) {
  const int b = c.cur;
  if (c.N == 0) return cudaSuccess;
  if (c.precision == RBE_FP64)
    gather_state_kernel<double><<<nblk(c.N, 256), 256, 0, c.stream>>>(s_id, v_id, c.id[b], c.N, c.s[b], c.vd[b]);
  else
    gather_state_kernel<float><<<nblk(c.N, 256), 256, 0, c.stream>>>(s_id, v_id, c.id[b], c.N, c.s[b], c.vf[b]);
  return cudaGetLastError();
}

void zero_partials_tail(Ctx &c, int64_t off, int64_t written, int64_t capacity) {
  if (written >= capacity) return;
  cudaMemsetAsync(c.epart + off + written * NQ_PAIR, 0,
                  sizeof(double) * (size_t)(capacity - written) * NQ_PAIR, c.stream);
}

cudaError_t launch_scatter_int(Ctx &c, const int32_t *src_sorted, int32_t *dst_id, int width) {
  const int b = c.cur;
  if (c.N == 0) return cudaSuccess;
  scatter_int_kernel<<<nblk(c.N, 256), 256, 0, c.stream>>>(src_sorted, c.id[b], c.N, width, dst_id);
  return cudaGetLastError();
}

}  // namespace rbe
