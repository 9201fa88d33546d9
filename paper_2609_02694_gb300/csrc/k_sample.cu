// k_sample.cu -- Philox counter-based importance sampler of the RBE modes (Eq. F_long_RBE).
//
// P i.i.d. modes k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z) from P(k) ~ exp(-k^2/4 alpha), k != 0.
// The density factorises over axes. Word d of one Philox4x32-10 block picks m_d by inverse
// CDF on the axis table (the host builds it once in FP64). m = 0 is rejected and redrawn
// with the next attempt counter. Mode l depends only on (seed, replica, step, l): every
// replica that knows the seed rebuilds the same ordered sample, which is the paper's
// seed-broadcast scheme (Sec. 2.3.1) with no communication.
// Integer work, one CTA, latency-bound; bit-exact with the FP64 oracle's draws.
#include <algorithm>

#include "rbe_internal.cuh"

namespace rbe {

struct SampleArgs {
  const uint64_t *T0, *T1, *T2;
  int M0, M1, M2;
  const uint64_t *step;
  uint2 key;
  int P;
  double tpx, tpy, tpz;  // 2 pi / L_d
  double cnum;           // 4 pi C S / (P V)
  int4 *m;
  float4 *kcf;
  double4_16a *kcd;
  int *err;
};

// Smallest i in [0, 2M] with w < T[i]; T[2M] = 2^32 so it exists.
__device__ __forceinline__ int inv_cdf(const uint64_t *T, int M, uint32_t w) {
  int lo = 0, hi = 2 * M;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (T[mid] > (uint64_t)w) hi = mid; else lo = mid + 1;
  }
  return lo - M;
}

// Axis tables of up to this many entries are searched from shared memory (24 KB for three).
constexpr int kSampleShared = 1024;

__device__ __forceinline__ void sample_k_body(const SampleArgs &a, int, int) {
  __shared__ uint64_t sT[3][kSampleShared];
  const uint32_t step = (uint32_t)(*a.step);
  // the binary searches' dependent loads from shared memory instead of L2 when they fit
  const bool fit = 2 * a.M0 + 1 <= kSampleShared && 2 * a.M1 + 1 <= kSampleShared &&
                   2 * a.M2 + 1 <= kSampleShared;
  const uint64_t *T0 = a.T0, *T1 = a.T1, *T2 = a.T2;
  if (fit) {
    for (int k = threadIdx.x; k <= 2 * a.M0; k += blockDim.x) sT[0][k] = a.T0[k];
    for (int k = threadIdx.x; k <= 2 * a.M1; k += blockDim.x) sT[1][k] = a.T1[k];
    for (int k = threadIdx.x; k <= 2 * a.M2; k += blockDim.x) sT[2][k] = a.T2[k];
    T0 = sT[0];
    T1 = sT[1];
    T2 = sT[2];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < a.P; l += blockDim.x) {
    int mx = 0, my = 0, mz = 0;
    bool ok = false;
    for (uint32_t attempt = 0; attempt < 64u && !ok; ++attempt) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)l, attempt, step, 0u), a.key);
      mx = inv_cdf(T0, a.M0, w.x);
      my = inv_cdf(T1, a.M1, w.y);
      mz = inv_cdf(T2, a.M2, w.z);
      ok = (mx | my | mz) != 0;
    }
    if (!ok) {
      atomicOr(a.err, ERRBIT_SAMPLER);
      mx = 1;  // keep the outputs finite; the host reports the flag
    }
    const double kx = a.tpx * mx, ky = a.tpy * my, kz = a.tpz * mz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    const double c = a.cnum / k2;
    a.m[l] = make_int4(mx, my, mz, 0);
    a.kcf[l] = make_float4((float)kx, (float)ky, (float)kz, (float)c);
    a.kcd[l] = make_double4_16a(kx, ky, kz, c);
  }
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), sample_k_kernel, SampleArgs, sample_k_body)

cudaError_t launch_sample_k(Ctx &c) {
  SampleArgs a;
  a.T0 = c.T[0]; a.T1 = c.T[1]; a.T2 = c.T[2];
  a.M0 = c.M[0]; a.M1 = c.M[1]; a.M2 = c.M[2];
  a.step = c.step_dev;
  a.key = make_uint2((uint32_t)c.seed, (uint32_t)(c.seed >> 32) ^ c.replica);
  a.P = c.P;
  a.tpx = 2.0 * kPi / c.box[0];
  a.tpy = 2.0 * kPi / c.box[1];
  a.tpz = 2.0 * kPi / c.box[2];
  a.cnum = 4.0 * kPi * c.C * c.S / ((double)c.P * c.V);
  a.m = c.m; a.kcf = c.kcf; a.kcd = c.kcd; a.err = c.err;
  return dispatch(c, sample_k_kernel, sample_k_kernel_b, dim3(1), dim3(256), 0, a);
}

__global__ void set_step_kernel(uint64_t *step_dev, uint64_t step) { *step_dev = step; }

struct StepArgs {
  uint64_t *step;
};
__device__ __forceinline__ void step_advance_body(const StepArgs &a, int, int) { *a.step += 1; }
RBE_BATCHED_KERNEL(, step_advance_kernel, StepArgs, step_advance_body)

// Zero n 32-bit words (grid-stride over the replica's own grid).
struct ZeroArgs {
  uint32_t *p;
  int64_t n;
};
__device__ __forceinline__ void zero_body(const ZeroArgs &a, int bx, int nbx) {
  for (int64_t k = (int64_t)bx * blockDim.x + threadIdx.x; k < a.n; k += (int64_t)nbx * blockDim.x)
    a.p[k] = 0u;
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), zero_kernel, ZeroArgs, zero_body)

cudaError_t fill_zero(Ctx &c, void *p, int64_t words) {
  if (words <= 0) return cudaSuccess;
  if (!c.rec) return cudaMemsetAsync(p, 0, sizeof(uint32_t) * (size_t)words, c.stream);
  ZeroArgs a{static_cast<uint32_t *>(p), words};
  const int64_t blocks = std::min<int64_t>((words + 255) / 256, 1024);
  return dispatch(c, zero_kernel, zero_kernel_b, dim3((unsigned)blocks), dim3(256), 0, a);
}

cudaError_t launch_set_step(Ctx &c, uint64_t step) {
  set_step_kernel<<<1, 1, 0, c.stream>>>(c.step_dev, step);
  return cudaGetLastError();
}

cudaError_t launch_step_advance(Ctx &c) {
  return dispatch(c, step_advance_kernel, step_advance_kernel_b, dim3(1), dim3(1), 0,
                  StepArgs{c.step_dev});
}

}  // namespace rbe
