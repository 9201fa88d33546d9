// rbe_noalloc.cu -- structure factor entry point that allocates no device memory.
//
// Some callers cannot allocate device memory. Examples: a host application that owns
// one fixed device pool and forbids libraries to allocate outside it, or a latency-bound
// loop in which the implicit device-wide synchronisation of cudaMalloc/cudaFree is not
// acceptable. rbe_structure_factor_noalloc serves them. The caller passes inputs and the
// output. The only scratch, the per-block partial sums, lives in the fixed-size
// file-scope device array below. Every GPU that loads the library holds that array
// until the process exits.
//
// The array is shared by every call on a device and keeps the last call's contents.
// Each call overwrites every partial slot it reads, so nothing needs clearing. Two
// calls whose work overlaps on the GPU (different streams, or different host threads
// with no ordering between them) race on the array.
#include <algorithm>
#include <mutex>

#include "rbe_internal.cuh"

namespace {

constexpr int64_t kNoallocScratchDoubles = (int64_t)1 << 20;  // 8 MiB of partial sums
constexpr int kNoallocMaxP = 65536;
constexpr int kNoallocThreads = 256;
constexpr int kNoallocTile = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocScratchDoubles];

std::mutex g_setup_mutex;
double *g_partials_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Block b sums tiles b, b + nblk, ... of the particles for one mode per thread, with
// Kahan-compensated FP32 accumulation (the compensated form of the handle path), and
// writes one partial per mode.
__global__ void __launch_bounds__(kNoallocThreads)
    noalloc_sf_kernel(const uint32_t *__restrict__ s, const float *__restrict__ q, int64_t N,
                      const int32_t *__restrict__ m, int P, int nblk,
                      double *__restrict__ part) {
  __shared__ uint4 sh[kNoallocTile];
  const int l = blockIdx.y * blockDim.x + threadIdx.x;
  int4 mm = make_int4(0, 0, 0, 0);
  if (l < P) mm = make_int4(m[3 * l], m[3 * l + 1], m[3 * l + 2], 0);
  float re = 0.f, im = 0.f, cre = 0.f, cim = 0.f;
  for (int64_t p0 = (int64_t)blockIdx.x * kNoallocTile; p0 < N;
       p0 += (int64_t)nblk * kNoallocTile) {
    const int np = (int)min((int64_t)kNoallocTile, N - p0);
    __syncthreads();
    for (int k = threadIdx.x; k < np; k += blockDim.x)
      sh[k] = make_uint4(s[p0 + k], s[N + p0 + k], s[2 * N + p0 + k], __float_as_uint(q[p0 + k]));
    __syncthreads();
    if (l < P) {
      for (int k = 0; k < np; ++k) {
        const uint4 e = sh[k];
        float sn, co;
        __sincosf(rbe::phase_to_radians(rbe::phase_u32(mm, e.x, e.y, e.z)), &sn, &co);
        const float qq = __uint_as_float(e.w);
        const float yr = fmaf(qq, co, -cre);
        const float tr = re + yr;
        cre = (tr - re) - yr;
        re = tr;
        const float yi = fmaf(qq, sn, -cim);
        const float ti = im + yi;
        cim = (ti - im) - yi;
        im = ti;
      }
    }
  }
  if (l < P) {
    double *out = part + ((int64_t)blockIdx.x * P + l) * 2;
    out[0] = (double)re - (double)cre;
    out[1] = (double)im - (double)cim;
  }
}

// One block per mode: fixed-order FP64 sum of the block partials.
__global__ void __launch_bounds__(128)
    noalloc_combine_kernel(const double *__restrict__ part, int nblk, int P,
                           double *__restrict__ rho) {
  __shared__ double sre[128], sim[128];
  const int l = blockIdx.x;
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    re += part[((int64_t)b * P + l) * 2];
    im += part[((int64_t)b * P + l) * 2 + 1];
  }
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int st = 64; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sre[threadIdx.x] += sre[threadIdx.x + st];
      sim[threadIdx.x] += sim[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rho[2 * l] = sre[0];
    rho[2 * l + 1] = sim[0];
  }
}

// Device address of the scratch array on the current device and that device's SM count,
// looked up once per device.
int partials_on_current_device(double **out, int *sms) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return RBE_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_ptr[dev]) {
    double *ptr = nullptr;
    if (cudaGetSymbolAddress((void **)&ptr, g_noalloc_partials) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return RBE_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      return RBE_ERR_CUDA;
    }
    g_sm_count[dev] = n;
    g_partials_ptr[dev] = ptr;
  }
  *out = g_partials_ptr[dev];
  *sms = g_sm_count[dev];
  return RBE_OK;
}

}  // namespace

extern "C" int rbe_structure_factor_noalloc(const uint32_t *s, const float *q, int64_t N,
                                            const int32_t *m, int P, double *rho,
                                            void *cuda_stream) {
  if (N < 0 || P < 1 || !m || !rho || (N > 0 && (!s || !q))) return RBE_ERR_INVALID;
  if (P > kNoallocMaxP) return RBE_ERR_INVALID;  // beyond the fixed scratch this build holds
  double *part = nullptr;
  int sms = 1;
  const int rc = partials_on_current_device(&part, &sms);
  if (rc != RBE_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int mode_blocks = (P + kNoallocThreads - 1) / kNoallocThreads;
  // as many particle blocks as the scratch holds for P modes, at most two per SM
  int64_t nblk = kNoallocScratchDoubles / (2 * (int64_t)P);
  nblk = std::min<int64_t>(nblk, 2 * (int64_t)sms);
  nblk = std::min<int64_t>(nblk, std::max<int64_t>(1, (N + kNoallocTile - 1) / kNoallocTile));
  nblk = std::max<int64_t>(nblk, 1);
  noalloc_sf_kernel<<<dim3((unsigned)nblk, (unsigned)mode_blocks), kNoallocThreads, 0, st>>>(
      s, q, N, m, P, (int)nblk, part);
  noalloc_combine_kernel<<<P, 128, 0, st>>>(part, (int)nblk, P, rho);
  if (cudaGetLastError() != cudaSuccess) return RBE_ERR_CUDA;
  return RBE_OK;
}
