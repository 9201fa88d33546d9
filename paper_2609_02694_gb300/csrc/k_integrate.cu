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
struct KickDriftArgs {
  V *v;
  const FT *F;
  const float *invm;
  uint32_t *s;
  int64_t N;
  double hdk, gx, gy, gz;
  int *err;
  const double *scale;
  uint64_t *step;  // the step counter, advanced by the first thread (the sampler reads it next)
};

// Solo and batched kernels of a body templated on the velocity and force types.
#define RBE_VF_KERNELS(LB, NAME, ARGS, BODY)                                                   \
  template <typename V, typename FT>                                                         \
  __global__ void LB NAME(const ARGS<V, FT> a) {                                              \
    BODY<V, FT>(a, (int)blockIdx.x, (int)gridDim.x);                                          \
  }                                                                                          \
  template <typename V, typename FT>                                                         \
  __global__ void LB NAME##_b(const ARGS<V, FT> *__restrict__ t,                              \
                              const int32_t *__restrict__ pre, int nrep) {                    \
    const BatchIdx q = batch_locate(pre, nrep);                                               \
    BODY<V, FT>(t[q.r], q.bx, q.nbx);                                                         \
  }

template <typename V, typename FT>
__device__ __forceinline__ void kick_drift_body(const KickDriftArgs<V, FT> &a, int bx, int) {
  const int64_t i = (int64_t)bx * blockDim.x + threadIdx.x;
  const int64_t N = a.N;
  if (i == 0) *a.step += 1;
  if (i >= N) return;
  V *__restrict__ v = a.v;
  const FT *__restrict__ F = a.F;
  uint32_t *__restrict__ s = a.s;
  const double *scale = a.scale;
  const double hdk = a.hdk;
  const double g[3] = {a.gx, a.gy, a.gz};
  const float *__restrict__ invm = a.invm;
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
  if (bad) atomicOr(a.err, ERRBIT_NONFINITE);
}
RBE_VF_KERNELS(__launch_bounds__(256), kick_drift_kernel, KickDriftArgs, kick_drift_body)

// The FP32 forms with N a multiple of 4: four consecutive particles a thread in 16-byte
// accesses (the arrays start 256-byte aligned, and d N keeps each axis block aligned), each
// with kick_drift_body's arithmetic in the same order.
__device__ __forceinline__ void kick_drift4_body(const KickDriftArgs<float, float> &a, int bx, int) {
  const int64_t q = (int64_t)bx * blockDim.x + threadIdx.x;
  const int64_t N = a.N;
  if (q == 0) *a.step += 1;
  const int64_t i = 4 * q;
  if (i >= N) return;
  const float4 im = *reinterpret_cast<const float4 *>(a.invm + i);
  const float sc = a.scale ? (float)*a.scale : 1.f;  // Nose-Hoover start-of-step scaling
  const float hdk = (float)a.hdk;
  const double g[3] = {a.gx, a.gy, a.gz};
  bool bad0 = false, bad1 = false, bad2 = false, bad3 = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float4 *vp = reinterpret_cast<float4 *>(a.v + d * N + i);
    uint4 *sp = reinterpret_cast<uint4 *>(a.s + d * N + i);
    float4 v = *vp;
    const float4 f = *reinterpret_cast<const float4 *>(a.F + d * N + i);
    uint4 sv = *sp;
    const float gd = (float)g[d];
    auto one = [&](float &vv, float ff, float imm, uint32_t &ss, bool &bad) {
      vv = vv * sc + ff * imm * hdk;
      const float inc = vv * gd;
      bad |= !isfinite(inc) || fabsf(inc) > 2.0e9f;
      const int st = bad ? 0 : __float2int_rn(inc);
      ss += (uint32_t)st;
    };
    one(v.x, f.x, im.x, sv.x, bad0);
    one(v.y, f.y, im.y, sv.y, bad1);
    one(v.z, f.z, im.z, sv.z, bad2);
    one(v.w, f.w, im.w, sv.w, bad3);
    *vp = v;
    *sp = sv;
  }
  if (bad0 || bad1 || bad2 || bad3) atomicOr(a.err, ERRBIT_NONFINITE);
}
using KickDriftArgsF = KickDriftArgs<float, float>;
RBE_BATCHED_KERNEL(__launch_bounds__(256), kick_drift4_kernel, KickDriftArgsF, kick_drift4_body)

template <typename V, typename FT>
struct KickArgs {
  V *v;
  const FT *F;
  const float *invm;
  int64_t N;
  double hdk, inv_kappa;
  int do_kick;
  double *ke_part;
};

template <typename V, typename FT>
__device__ __forceinline__ void kick_body(const KickArgs<V, FT> &a, int bx, int) {
  __shared__ double sh[256];
  V *__restrict__ v = a.v;
  const FT *__restrict__ F = a.F;
  const float *__restrict__ invm = a.invm;
  const int64_t N = a.N;
  const double hdk = a.hdk, inv_kappa = a.inv_kappa;
  const int do_kick = a.do_kick;
  const int64_t i = (int64_t)bx * blockDim.x + threadIdx.x;
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
  if (threadIdx.x == 0) a.ke_part[bx] = sh[0];
}
RBE_VF_KERNELS(__launch_bounds__(256), kick_kernel, KickArgs, kick_body)

// The FP32 forms with N a multiple of 4: blocks of 64 threads over the same 256 particles as
// kick_body's blocks, four consecutive particles a thread in 16-byte accesses. Each particle's
// arithmetic, its term's shared-memory slot and the reduction tree are kick_body's, so the
// kinetic energy partials are the same bit for bit.
__device__ __forceinline__ void kick4_body(const KickArgs<float, float> &a, int bx, int) {
  __shared__ double sh[256];
  const int64_t N = a.N;
  const int t = threadIdx.x;
  const int64_t i = (int64_t)bx * 256 + 4 * t;
  const float hdk = (float)a.hdk, ik = (float)a.inv_kappa;
  double ke[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < N) {  // (all four, N being a multiple of 4)
    const float4 im = *reinterpret_cast<const float4 *>(a.invm + i);
    float v2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float4 *vp = reinterpret_cast<float4 *>(a.v + d * N + i);
      float4 vv = *vp;
      if (a.do_kick) {
        const float4 f = *reinterpret_cast<const float4 *>(a.F + d * N + i);
        vv.x += f.x * im.x * hdk;
        vv.y += f.y * im.y * hdk;
        vv.z += f.z * im.z * hdk;
        vv.w += f.w * im.w * hdk;
        *vp = vv;
      }
      v2[0] += vv.x * vv.x;
      v2[1] += vv.y * vv.y;
      v2[2] += vv.z * vv.z;
      v2[3] += vv.w * vv.w;
    }
    ke[0] = (double)(0.5f * v2[0] * __frcp_rn(im.x) * ik);
    ke[1] = (double)(0.5f * v2[1] * __frcp_rn(im.y) * ik);
    ke[2] = (double)(0.5f * v2[2] * __frcp_rn(im.z) * ik);
    ke[3] = (double)(0.5f * v2[3] * __frcp_rn(im.w) * ik);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sh[4 * t + j] = ke[j];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    for (int k = t; k < st; k += 64) sh[k] += sh[k + st];
    __syncthreads();
  }
  if (t == 0) a.ke_part[bx] = sh[0];
}
using KickArgsF = KickArgs<float, float>;
RBE_BATCHED_KERNEL(__launch_bounds__(64), kick4_kernel, KickArgsF, kick4_body)

// Nose-Hoover half steps (chain of one): from 2K = 2 sum(kinetic partials) the end-of-step
// half (mode 0) gives the velocity scale s_end and the start-of-next-step half gives
// s_start, applied by the next kick-drift; mode 1 only does the start half (first step).
struct ThermoArgs {
  const double *ke_part;
  int64_t n;
  double Nf, kT, Q, dt;
  double *th;
  int mode;
};

__device__ __forceinline__ void thermostat_body(const ThermoArgs &a, int, int) {
  __shared__ double sh[256];
  const double *__restrict__ ke_part = a.ke_part;
  const int64_t n = a.n;
  const double Nf = a.Nf, kT = a.kT, Q = a.Q, dt = a.dt;
  double *__restrict__ th = a.th;
  const int mode = a.mode;
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
RBE_BATCHED_KERNEL(__launch_bounds__(256), thermostat_kernel, ThermoArgs, thermostat_body)

template <typename V, typename FT>
struct ScaleArgs {
  V *v;
  int64_t N;
  const double *scale;
};
template <typename V, typename FT>
__device__ __forceinline__ void scale_v_body(const ScaleArgs<V, FT> &a, int bx, int) {
  const int64_t k = (int64_t)bx * blockDim.x + threadIdx.x;
  if (k >= 3 * a.N) return;
  a.v[k] *= (V)*a.scale;
}
RBE_VF_KERNELS(__launch_bounds__(256), scale_v_kernel, ScaleArgs, scale_v_body)

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
// partials in flight per thread), then warp shuffles, then the warp sums in order. Four
// warps: the warp reductions of seven FP64 sums dominate on one SM (FP64 runs at 1/64 of the
// FP32 rate), and they scale with the warps, the strided sums do not.
constexpr int kTotalsThreads = 128;

template <typename ACC>
__device__ __forceinline__ void totals_body(const TotalsArgs &a, int, int) {
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
template <typename ACC>
__global__ void __launch_bounds__(kTotalsThreads) totals_kernel(const TotalsArgs a) {
  totals_body<ACC>(a, (int)blockIdx.x, (int)gridDim.x);
}
template <typename ACC>
__global__ void __launch_bounds__(kTotalsThreads)
    totals_kernel_b(const TotalsArgs *__restrict__ t, const int32_t *__restrict__ pre, int nrep) {
  const BatchIdx q = batch_locate(pre, nrep);
  totals_body<ACC>(t[q.r], q.bx, q.nbx);
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

// First half-kick and drift, with the step counter's advance (alone when there are no
// particles).
cudaError_t launch_kick_drift(Ctx &c) {
  const int b = c.cur;
  const double hdk = 0.5 * c.dt * c.kappa;
  if (c.N == 0) return launch_step_advance(c);
  const double *scale = c.nvt ? c.thermo + 2 : nullptr;
  const double gx = c.dt * kTwo32 / c.box[0], gy = c.dt * kTwo32 / c.box[1],
               gz = c.dt * kTwo32 / c.box[2];
  const dim3 g(nblk(c.N, 256)), t(256);
  if (c.precision == RBE_FP64) {
    const KickDriftArgs<double, double> a{c.vd[b], c.Fd, c.invm[b], c.s[b], c.N, hdk, gx, gy, gz,
                                          c.err, scale, c.step_dev};
    return dispatch(c, kick_drift_kernel<double, double>, kick_drift_kernel_b<double, double>, g,
                    t, 0, a);
  }
  const KickDriftArgs<float, float> a{c.vf[b], c.F, c.invm[b], c.s[b], c.N, hdk, gx, gy, gz,
                                      c.err, scale, c.step_dev};
  // (a batch keeps the one-particle kernel: the same results, and replicas of any N share a
  //  class)
  if (c.N % 4 == 0 && !c.rec)
    return dispatch(c, kick_drift4_kernel, kick_drift4_kernel_b, dim3(nblk(c.N / 4, 256)), t, 0,
                    a);
  return dispatch(c, kick_drift_kernel<float, float>, kick_drift_kernel_b<float, float>, g, t, 0,
                  a);
}

cudaError_t launch_thermostat(Ctx &c, int mode) {
  const int b = c.cur;
  const ThermoArgs ta{c.epart + c.off_ke, c.n_ke_blk, c.Nf, c.kB * c.T0, c.Qnh, c.dt, c.thermo,
                      mode};
  cudaError_t e = dispatch(c, thermostat_kernel, thermostat_kernel_b, dim3(1), dim3(256), 0, ta);
  if (e != cudaSuccess || mode != 0) return e;
  const dim3 g(nblk(3 * c.N, 256)), t(256);
  if (c.precision == RBE_FP64) {
    const ScaleArgs<double, double> a{c.vd[b], c.N, c.thermo + 4};
    return dispatch(c, scale_v_kernel<double, double>, scale_v_kernel_b<double, double>, g, t, 0, a);
  }
  const ScaleArgs<float, float> a{c.vf[b], c.N, c.thermo + 4};
  return dispatch(c, scale_v_kernel<float, float>, scale_v_kernel_b<float, float>, g, t, 0, a);
}

static cudaError_t kick_impl(Ctx &c, int do_kick) {
  const int b = c.cur;
  const double hdk = 0.5 * c.dt * c.kappa;
  if (c.N == 0) return cudaSuccess;
  const dim3 g(nblk(c.N, 256)), t(256);
  if (c.precision == RBE_FP64) {
    const KickArgs<double, double> a{c.vd[b], c.Fd, c.invm[b], c.N, hdk, 1.0 / c.kappa, do_kick,
                                     c.epart + c.off_ke};
    return dispatch(c, kick_kernel<double, double>, kick_kernel_b<double, double>, g, t, 0, a);
  }
  const KickArgs<float, float> a{c.vf[b], c.F, c.invm[b], c.N, hdk, 1.0 / c.kappa, do_kick,
                                 c.epart + c.off_ke};
  // (a batch keeps the one-particle kernel: the same results, and replicas of any N share a
  //  class)
  if (c.N % 4 == 0 && !c.rec) return dispatch(c, kick4_kernel, kick4_kernel_b, g, dim3(64), 0, a);
  return dispatch(c, kick_kernel<float, float>, kick_kernel_b<float, float>, g, t, 0, a);
}

cudaError_t launch_kick(Ctx &c) { return kick_impl(c, 1); }
cudaError_t launch_kinetic(Ctx &c) { return kick_impl(c, 0); }

// Block partials of a pair pass ([nblk][NQ_PAIR]) summed over fixed contiguous ranges in a
// fixed order into [gridDim.x][NQ_PAIR]: the FP64 adds are spread over many SMs (one SM's
// FP64 rate is low) before the one-block totals.
struct CompactArgs {
  const double *in;
  int64_t nblk, per;
  double *out;
};

__device__ __forceinline__ void partials_compact_body(const CompactArgs &a, int bx, int) {
  __shared__ double sh[NQ_PAIR][256];
  const double *__restrict__ in = a.in;
  const int64_t nblk = a.nblk, per = a.per;
  const int64_t b0 = (int64_t)bx * per, b1 = min(nblk, b0 + per);
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
  if (threadIdx.x < NQ_PAIR) a.out[(int64_t)bx * NQ_PAIR + threadIdx.x] = sh[threadIdx.x][0];
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), partials_compact_kernel, CompactArgs,
                   partials_compact_body)

int64_t partials_compact_count(int64_t nblk) { return std::min<int64_t>(nblk, kCompactMax); }

cudaError_t launch_totals(Ctx &c) {
  TotalsArgs a;
  // pair and Coulomb-pass partials, compacted first (at most kCompactMax per pass)
  const int64_t ncp = partials_compact_count(c.n_pair_blk), ncc = partials_compact_count(c.n_coul_blk);
  cudaError_t e;
  if (ncp > 0) {
    const CompactArgs ca{c.epart + c.off_pair, c.n_pair_blk, (c.n_pair_blk + ncp - 1) / ncp,
                         c.ecomp};
    e = dispatch(c, partials_compact_kernel, partials_compact_kernel_b, dim3((unsigned)ncp),
                 dim3(256), 0, ca);
    if (e != cudaSuccess) return e;
  }
  if (ncc > 0) {
    const CompactArgs ca{c.epart + c.off_coul, c.n_coul_blk, (c.n_coul_blk + ncc - 1) / ncc,
                         c.ecomp + kCompactMax * NQ_PAIR};
    e = dispatch(c, partials_compact_kernel, partials_compact_kernel_b, dim3((unsigned)ncc),
                 dim3(256), 0, ca);
    if (e != cudaSuccess) return e;
  }
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
  if (c.precision == RBE_FP32)
    return dispatch(c, totals_kernel<float>, totals_kernel_b<float>, dim3(1), dim3(kTotalsThreads),
                    0, a);
  return dispatch(c, totals_kernel<double>, totals_kernel_b<double>, dim3(1),
                  dim3(kTotalsThreads), 0, a);
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
  fill_zero(c, c.epart + off + written * NQ_PAIR, 2 * (capacity - written) * NQ_PAIR);
}

cudaError_t launch_scatter_int(Ctx &c, const int32_t *src_sorted, int32_t *dst_id, int width) {
  const int b = c.cur;
  if (c.N == 0) return cudaSuccess;
  scatter_int_kernel<<<nblk(c.N, 256), 256, 0, c.stream>>>(src_sorted, c.id[b], c.N, width, dst_id);
  return cudaGetLastError();
}

}  // namespace rbe
