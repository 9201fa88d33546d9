// k_probe.cu -- throughput probes that supply the roofline denominators the driver does not
// measure (FP32 FMA, SFU sine/cosine, FP64 FMA). Each probe runs 8 independent dependency
// chains per thread on every SM (16 resident blocks of 256 threads per SM) and is timed with
// CUDA events; the host reports operations per second at the clock the GPU ran at.
#include "rbe_internal.cuh"

namespace rbe {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) probe_fp32_kernel(float a, float b, int iters,
                                                                  float *out) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = a + (float)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], b, a);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1.2345f) out[0] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(kProbeThreads) probe_sincos_kernel(float a, int iters,
                                                                    float *out) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = a * (float)(threadIdx.x + k + 1);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float sn, co;
      __sincosf(x[k], &sn, &co);
      x[k] = sn + co;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1.2345f) out[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_fp64_kernel(double a, double b, int iters,
                                                                  double *out) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = a + (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], b, a);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1.2345) out[0] = s;
}

}  // namespace rbe

using namespace rbe;

extern "C" int rbe_measure_peak(int kind, double *ops_per_s, double *ms_out) {
  if (!ops_per_s || kind < 0 || kind > 2) return RBE_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return RBE_ERR_CUDA;
  }
  void *buf = nullptr;
  if (cudaMalloc(&buf, 64) != cudaSuccess) { cudaGetLastError(); return RBE_ERR_OOM; }
  const int blocks = sms * 16;
  const int iters = kind == 2 ? 512 : 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // first launch warms up
    cudaEventRecord(e0);
    if (kind == 0) probe_fp32_kernel<<<blocks, kProbeThreads>>>(1.0001f, 0.9999f, iters, (float *)buf);
    else if (kind == 1) probe_sincos_kernel<<<blocks, kProbeThreads>>>(0.001f, iters, (float *)buf);
    else probe_fp64_kernel<<<blocks, kProbeThreads>>>(1.0001, 0.9999, iters, (double *)buf);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (cudaGetLastError() != cudaSuccess) return RBE_ERR_CUDA;
  const double threads = (double)blocks * kProbeThreads;
  const double ops = threads * 8.0 * iters * (kind == 1 ? 1.0 : 2.0);  // FMA = 2 flops
  *ops_per_s = ops / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return RBE_OK;
}
