// k_kspace.cu -- structure factor and k-space force gather of the RBE estimator.
//
// rho(k_l) = sum_j q_j exp(i k_l . r_j)           (Eq. U_Coul_Fourier, charged particles only)
// F_i = -q_i sum_l c_l k_l (Im rho_l cos t_il - Re rho_l sin t_il),  c_l = 4 pi C S / (P V k_l^2)
//                                                  (Eq. F_long_RBE with the sign of Eq. F_i)
// U = sum_l (c_l / 2) |rho_l|^2,  W = sum_l (c_l / 2) |rho_l|^2 (1 - k_l^2 / 2 alpha)
//
// Phases are exact: on the 2^-32 grid k_l . r_j / 2 pi = sum_d m_d s_d / 2^32 (mod 1), an
// integer multiply-add in wrapping uint32 arithmetic. Only the final angle is rounded
// (2^-23 turns in the FP32 forms).
//
// The paper's pipeline is sampling -> local accumulation -> global reduction ->
// force application (Sec. 2.3.1). On one GPU its AllReduce of 2P values becomes a grid
// reduction. Each block writes compensated FP32 partials of its particle tile for a
// contiguous slice of modes (one thread per mode, particles broadcast from shared memory,
// no atomics). A combine kernel then sums the partials in FP64 in a fixed order, so the
// result is reproducible run to run. Both passes are bound by the SFU (one sincos per
// particle and mode) and FP32/INT issue.
#include "rbe_internal.cuh"

namespace rbe {

struct SfArgs {
  const uint32_t *cs;
  const float *cqf;
  const double *cqd;
  int64_t Nq;
  const int4 *m;
  int P, tile;
  double *part;
};
struct CombineArgs {
  const double *part;
  int nblk, P;
  const double4_16a *kcd;
  double alpha;
  double2 *rho;
  float2 *abf;
  double2 *abd;
  double *emode;
};
struct GatherArgs {
  const uint32_t *cs;
  const float *cqf;
  const double *cqd;
  int64_t Nq;
  const int4 *m;
  const float4 *kcf;
  const double4_16a *kcd;
  const float2 *abf;
  const double2 *abd;
  int P;
  const int32_t *cmap;
  float *F;
  double *Fd;
  int64_t N;
  long long *facc;         // nullable: add to these 3 x N fixed-point sums instead of F
  float fscale;            // (their scale in the FP32 forms,
  double fscale_d;         //  and in the FP64 form)
  int *err;
};

// Solo and batched kernels of a body templated on MODE.
#define RBE_MODE_KERNELS(LB, NAME, ARGS, BODY)                                                 \
  template <int MODE>                                                                        \
  __global__ void LB NAME(const ARGS a) { BODY<MODE>(a, (int)blockIdx.x, (int)gridDim.x); }   \
  template <int MODE>                                                                        \
  __global__ void LB NAME##_b(const ARGS *__restrict__ t, const int32_t *__restrict__ pre,   \
                              int nrep) {                                                     \
    const BatchIdx q = batch_locate(pre, nrep);                                               \
    BODY<MODE>(t[q.r], q.bx, q.nbx);                                                          \
  }

// MODE: 0 = FP32 with Kahan-compensated per-thread sums, 1 = plain FP32, 2 = FP64.
template <int MODE>
__device__ __forceinline__ void sf_body(const SfArgs &a, int bx, int) {
  extern __shared__ uint4 sh[];
  const uint32_t *__restrict__ cs = a.cs;
  const float *__restrict__ cqf = a.cqf;
  const double *__restrict__ cqd = a.cqd;
  const int64_t Nq = a.Nq;
  const int P = a.P, tile = a.tile;
  const int64_t p0 = (int64_t)bx * tile;
  const int np = (int)min((int64_t)tile, Nq - p0);
  double *shq = reinterpret_cast<double *>(sh + tile);
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    sh[k] = make_uint4(cs[p0 + k], cs[Nq + p0 + k], cs[2 * Nq + p0 + k],
                       __float_as_uint(cqf[p0 + k]));
    if (MODE == 2) shq[k] = cqd[p0 + k];
  }
  __syncthreads();
  const int l = blockIdx.y * blockDim.x + threadIdx.x;
  if (l >= P) return;
  const int4 mm = a.m[l];
  double *out = a.part + ((int64_t)bx * P + l) * 2;
  if (MODE == 2) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < np; ++k) {
      const uint4 e = sh[k];
      double sn, co;
      sincos(phase_to_radians_d(phase_u32(mm, e.x, e.y, e.z)), &sn, &co);
      re = mad(shq[k], co, re);
      im = mad(shq[k], sn, im);
    }
    out[0] = re;
    out[1] = im;
  } else {
    float re = 0.f, im = 0.f, cre = 0.f, cim = 0.f;
    for (int k = 0; k < np; ++k) {
      const uint4 e = sh[k];
      float sn, co;
      __sincosf(phase_to_radians(phase_u32(mm, e.x, e.y, e.z)), &sn, &co);
      const float q = __uint_as_float(e.w);
      if (MODE == 0) {  // Kahan summation
        const float yr = fmaf(q, co, -cre);
        const float tr = re + yr;
        cre = (tr - re) - yr;
        re = tr;
        const float yi = fmaf(q, sn, -cim);
        const float ti = im + yi;
        cim = (ti - im) - yi;
        im = ti;
      } else {
        re = fmaf(q, co, re);
        im = fmaf(q, sn, im);
      }
    }
    out[0] = (double)re - (double)cre;
    out[1] = (double)im - (double)cim;
  }
}
RBE_MODE_KERNELS(__launch_bounds__(256), sf_kernel, SfArgs, sf_body)

// One block per mode: sum the block partials in a fixed order, then derive the per-mode
// energy, virial and the gather coefficients (c Im rho, c Re rho).
template <int MODE>
__device__ __forceinline__ void sf_combine_body(const CombineArgs &a, int bx, int) {
  __shared__ double sre[128], sim[128];
  __shared__ float fre[128], fim[128];
  const double *__restrict__ part = a.part;
  const int nblk = a.nblk, P = a.P;
  const int l = bx;
  if (MODE == 1) {
    float re = 0.f, im = 0.f;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      re += (float)part[((int64_t)b * P + l) * 2];
      im += (float)part[((int64_t)b * P + l) * 2 + 1];
    }
    fre[threadIdx.x] = re;
    fim[threadIdx.x] = im;
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        fre[threadIdx.x] += fre[threadIdx.x + s];
        fim[threadIdx.x] += fim[threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) { sre[0] = fre[0]; sim[0] = fim[0]; }
  } else {
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      re += part[((int64_t)b * P + l) * 2];
      im += part[((int64_t)b * P + l) * 2 + 1];
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        sre[threadIdx.x] += sre[threadIdx.x + s];
        sim[threadIdx.x] += sim[threadIdx.x + s];
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    const double re = sre[0], im = sim[0];
    const double4_16a kc = a.kcd[l];
    const double k2 = kc.x * kc.x + kc.y * kc.y + kc.z * kc.z;
    const double E = 0.5 * kc.w * (re * re + im * im);
    a.rho[l] = make_double2(re, im);
    a.emode[2 * l] = E;
    a.emode[2 * l + 1] = E * (1.0 - k2 / (2.0 * a.alpha));
    a.abf[l] = make_float2((float)(kc.w * im), (float)(kc.w * re));
    a.abd[l] = make_double2(kc.w * im, kc.w * re);
  }
}
RBE_MODE_KERNELS(__launch_bounds__(128), sf_combine_kernel, CombineArgs, sf_combine_body)

constexpr int kGatherThreads = 256;
constexpr int kGatherChunk = 256;

template <int MODE>
__device__ __forceinline__ void gather_body(const GatherArgs &a, int bx, int) {
  const uint32_t *__restrict__ cs = a.cs;
  const int64_t Nq = a.Nq, N = a.N;
  const int P = a.P;
  const int4 *__restrict__ m = a.m;
  const float4 *__restrict__ kcf = a.kcf;
  const double4_16a *__restrict__ kcd = a.kcd;
  const float2 *__restrict__ abf = a.abf;
  const double2 *__restrict__ abd = a.abd;
  __shared__ int4 sm[kGatherChunk];
  __shared__ float4 skf[kGatherChunk];
  __shared__ float2 sabf[kGatherChunk];
  __shared__ double4_16a skd[MODE == 2 ? kGatherChunk : 1];
  __shared__ double2 sabd[MODE == 2 ? kGatherChunk : 1];
  const int64_t i = (int64_t)bx * blockDim.x + threadIdx.x;
  const bool valid = i < Nq;
  const uint32_t sx = valid ? cs[i] : 0u, sy = valid ? cs[Nq + i] : 0u,
                 sz = valid ? cs[2 * Nq + i] : 0u;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  double dx = 0.0, dy = 0.0, dz = 0.0;
  for (int l0 = 0; l0 < P; l0 += kGatherChunk) {
    const int nl = min(kGatherChunk, P - l0);
    __syncthreads();
    for (int t = threadIdx.x; t < nl; t += blockDim.x) {
      sm[t] = m[l0 + t];
      if (MODE == 2) {
        skd[t] = kcd[l0 + t];
        sabd[t] = abd[l0 + t];
      } else {
        skf[t] = kcf[l0 + t];
        sabf[t] = abf[l0 + t];
      }
    }
    __syncthreads();
    if (MODE == 2) {
      for (int t = 0; t < nl; ++t) {
        double sn, co;
        sincos(phase_to_radians_d(phase_u32(sm[t], sx, sy, sz)), &sn, &co);
        const double g = mad(sabd[t].x, co, -(sabd[t].y * sn));
        dx = mad(g, skd[t].x, dx);
        dy = mad(g, skd[t].y, dy);
        dz = mad(g, skd[t].z, dz);
      }
    } else {
      for (int t = 0; t < nl; ++t) {
        float sn, co;
        __sincosf(phase_to_radians(phase_u32(sm[t], sx, sy, sz)), &sn, &co);
        const float g = mad(sabf[t].x, co, -(sabf[t].y * sn));
        fx = fmaf(g, skf[t].x, fx);
        fy = fmaf(g, skf[t].y, fy);
        fz = fmaf(g, skf[t].z, fz);
      }
    }
  }
  if (!valid) return;
  const int64_t p = a.cmap[i];
  if (a.facc) {  // into the cluster kernel's fixed-point sums (integer atomics)
    if (MODE == 2) {
      const double q = a.cqd[i];
      fx_add(a.facc + p, -q * dx, a.fscale_d, a.err);
      fx_add(a.facc + N + p, -q * dy, a.fscale_d, a.err);
      fx_add(a.facc + 2 * N + p, -q * dz, a.fscale_d, a.err);
    } else {
      const float q = a.cqf[i];
      fx_add_i32(a.facc + p, -q * fx, a.fscale, a.err);
      fx_add_i32(a.facc + N + p, -q * fy, a.fscale, a.err);
      fx_add_i32(a.facc + 2 * N + p, -q * fz, a.fscale, a.err);
    }
  } else if (MODE == 2) {
    double *__restrict__ Fd = a.Fd;
    const double q = a.cqd[i];
    Fd[p] = mad(-q, dx, Fd[p]);
    Fd[N + p] = mad(-q, dy, Fd[N + p]);
    Fd[2 * N + p] = mad(-q, dz, Fd[2 * N + p]);
  } else {
    float *__restrict__ F = a.F;
    const float q = a.cqf[i];
    F[p] = mad(-q, fx, F[p]);
    F[N + p] = mad(-q, fy, F[N + p]);
    F[2 * N + p] = mad(-q, fz, F[2 * N + p]);
  }
}
RBE_MODE_KERNELS(__launch_bounds__(kGatherThreads), gather_kernel, GatherArgs, gather_body)

template <int MODE>
static cudaError_t sf_launch(Ctx &c, dim3 grid, size_t shm) {
  const SfArgs a{c.cs, c.cqf, c.cqd, c.Nq, c.m, c.P, c.sf_tile, c.sf_part};
  cudaError_t e = dispatch(c, sf_kernel<MODE>, sf_kernel_b<MODE>, grid, dim3(c.sf_mb), shm, a);
  if (e != cudaSuccess) return e;
  const CombineArgs b{c.sf_part, c.sf_nblk_p, c.P, c.kcd, c.alpha, c.rho, c.abf, c.abd, c.emode};
  return dispatch(c, sf_combine_kernel<MODE>, sf_combine_kernel_b<MODE>, dim3(c.P), dim3(128),
                  0, b);
}

cudaError_t launch_structure_factor(Ctx &c) {
  if (c.Nq == 0) return cudaSuccess;
  const dim3 grid((unsigned)c.sf_nblk_p, (unsigned)c.sf_nblk_m);
  const size_t shm = (size_t)c.sf_tile * (sizeof(uint4) + (c.precision == RBE_FP64 ? 8 : 0));
  switch (c.precision) {
    case RBE_FP32_COMP: return sf_launch<0>(c, grid, shm);
    case RBE_FP32: return sf_launch<1>(c, grid, shm);
    default: return sf_launch<2>(c, grid, shm);
  }
}

cudaError_t launch_kspace_gather(Ctx &c, bool into_facc) {
  if (c.Nq == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((c.Nq + kGatherThreads - 1) / kGatherThreads);
  const GatherArgs a{c.cs, c.cqf, c.cqd, c.Nq, c.m, c.kcf, c.kcd, c.abf, c.abd, c.P, c.cmap,
                     c.F, c.Fd, c.N, into_facc ? c.facc : nullptr, (float)kFixScale32,
                     kFixScale64, c.err};
  // (into the fixed-point sums it runs per replica in a batch, within the pair pass's run)
  if (c.precision == RBE_FP64)
    return dispatch(c, gather_kernel<2>, gather_kernel_b<2>, dim3(blocks), dim3(kGatherThreads),
                    0, a, into_facc);
  return dispatch(c, gather_kernel<0>, gather_kernel_b<0>, dim3(blocks), dim3(kGatherThreads), 0,
                  a, into_facc);
}

}  // namespace rbe
