// k_sample.cu -- Philox counter-based importance sampler of the RBE modes (Eq. F_long_RBE).
//
// P i.i.d. modes k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z) from P(k) ~ exp(-k^2/4 alpha), k != 0.
// The density factorises over axes. Word d of one Philox4x32-10 block picks m_d by inverse
// CDF on the axis table (the host builds it once in FP64). m = 0 is rejected and redrawn
// with the next attempt counter. Mode l depends only on (seed, replica, step, l): every
// replica that knows the seed rebuilds the same ordered sample, which is the paper's
// seed-broadcast scheme (Sec. 2.3.1) with no communication.
// Integer work, one CTA, latency-bound; bit-exact with the FP64 oracle's draws.
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

__global__ void __launch_bounds__(256) sample_k_kernel(SampleArgs a) {
  const uint32_t step = (uint32_t)(*a.step);
  for (int l = threadIdx.x; l < a.P; l += blockDim.x) {
    int mx = 0, my = 0, mz = 0;
    bool ok = false;
    for (uint32_t attempt = 0; attempt < 64u && !ok; ++attempt) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)l, attempt, step, 0u), a.key);
      mx = inv_cdf(a.T0, a.M0, w.x);
      my = inv_cdf(a.T1, a.M1, w.y);
      mz = inv_cdf(a.T2, a.M2, w.z);
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
  sample_k_kernel<<<1, 256, 0, c.stream>>>(a);
  return cudaGetLastError();
}

__global__ void set_step_kernel(uint64_t *step_dev, uint64_t step) { *step_dev = step; }
__global__ void step_advance_kernel(uint64_t *step_dev) { *step_dev += 1; }

cudaError_t launch_set_step(Ctx &c, uint64_t step) {
  set_step_kernel<<<1, 1, 0, c.stream>>>(c.step_dev, step);
  return cudaGetLastError();
}

cudaError_t launch_step_advance(Ctx &c) {
  step_advance_kernel<<<1, 1, 0, c.stream>>>(c.step_dev);
  return cudaGetLastError();
}

}  // namespace rbe
