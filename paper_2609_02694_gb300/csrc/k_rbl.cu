// k_rbl.cu -- random batch list short-range force (Eqs. Ci_Si, RBL, F_corr).
//
// For each particle i, with cells of side >= r_s:
//   C_i = {j != i: r_ij <= r_core}, S_i = {j: r_core < r_ij <= r_s}
//   F~_i = sum_{C_i} F_ij + (#S_i / p) sum_{B_i} F_ij,  B_i = p i.i.d. uniform draws from S_i
//   F_i  = F~_i - (1/N) sum_j F~_j
// (The paper's core cutoff r_c is `r_core` here and its r_s is the real-space cutoff.)
// S_i is enumerated in a canonical order shared with the oracle: the 27 neighbour cells
// in (dz, dy, dx) order, each offset from -1 to 1, and inside each cell the (cell, id)
// order of the binning. Draw t takes idx = floor(w * #S_i / 2^32), where w is word
// (t mod 4) of Philox4x32-10 with counter (id_i, t / 4, step, 1). When #S_i <= p the whole
// shell enters with weight 1.
//
// Work decomposition: one thread per i. Lanes of a warp that share a cell walk that
// cell's 27 neighbours together. Candidates are staged in shared memory in FP32
// coordinates relative to the group leader. Membership is decided exactly: FP32 outside
// a +-1e-5 band around r_core^2 and r_s^2, the FP64 oracle expression inside it.
// Pass 1 counts #S_i and queues core pairs, which are evaluated from exact integer
// displacements. Pass 2 walks the same order again and evaluates the drawn shell pairs.
// The mean-force correction is a fixed-order FP64 reduction followed by a subtraction.
#include <climits>

#include "pair_common.cuh"

namespace rbe {

constexpr int kRblWarps = 4;
constexpr int kRblMaxP = 32;

struct RblArgs {
  PairArgs pa;
  const int32_t *id;
  float rcore2_lo, rcore2_hi, rs2_lo, rs2_hi;
  double rcore2d, rs2d;
  int p;
  uint2 key;
  const uint64_t *step;
  double *fsum_part;   // per block: sum of F~ (3 doubles)
  int32_t *ncore, *nshell, *partners;  // sorted order, nullable
};

// 0: outside r_s, 1: core, 2: shell. Exact at both radii.
__device__ __forceinline__ int rbl_classify(const RblArgs &a, float r2, uint32_t sxi, uint32_t syi,
                                            uint32_t szi, int64_t j) {
  if (r2 < a.rcore2_lo) return 1;
  if (r2 > a.rs2_hi) return 0;
  if (r2 > a.rcore2_hi && r2 < a.rs2_lo) return 2;
  const double e2 = exact_r2(a.pa.pc, (int)(sxi - a.pa.set.sx[j]), (int)(syi - a.pa.set.sy[j]),
                             (int)(szi - a.pa.set.sz[j]));
  if (e2 <= a.rcore2d) return 1;
  if (e2 <= a.rs2d) return 2;
  return 0;
}

template <typename real, bool COUL, bool MULTI>
__device__ __forceinline__ void rbl_pair(const RblArgs &a, const LJTable *tab, uint32_t sxi,
                                         uint32_t syi, uint32_t szi, real qi, int ti, int64_t j,
                                         PairAcc<real> &acc) {
  const PairConst &pc = a.pa.pc;
  const int dsx = (int)(sxi - a.pa.set.sx[j]);
  const int dsy = (int)(syi - a.pa.set.sy[j]);
  const int dsz = (int)(szi - a.pa.set.sz[j]);
  real dx, dy, dz;
  if (sizeof(real) == 8) {
    dx = (real)((double)dsx * pc.hd[0]); dy = (real)((double)dsy * pc.hd[1]); dz = (real)((double)dsz * pc.hd[2]);
  } else {
    dx = (real)((float)dsx * pc.h[0]); dy = (real)((float)dsy * pc.h[1]); dz = (real)((float)dsz * pc.h[2]);
  }
  const real r2 = dx * dx + dy * dy + dz * dz;
  pair_force<real, true, COUL, MULTI>(a.pa, tab, dx, dy, dz, r2, qi, ti, j, acc);
}

template <typename real, bool COUL, bool MULTI, bool WRAP>
__global__ void __launch_bounds__(kRblWarps * 32) rbl_kernel(const RblArgs a) {
  __shared__ float4 stage[kRblWarps][32];
  __shared__ int32_t list[kRblWarps][kListK][32];
  __shared__ double wred[kRblWarps][NQ_PAIR + 3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const PairSet &S = a.pa.set;
  const int64_t n = S.n;
  const int64_t i0 = ((int64_t)blockIdx.x * kRblWarps + wid) * 32;
  const int64_t i = i0 + lane;
  const bool valid = i < n;
  const LJTable *tab = a.pa.table;
  PairAcc<real> core, shell;
  core.fx = core.fy = core.fz = core.ulj = core.wlj = core.uc = core.wc = (real)0;
  core.cuc = core.cwc = (real)0;
  shell = core;
  core.nbr = shell.nbr = 0;
  real fx = 0, fy = 0, fz = 0;
  double en[NQ_PAIR] = {0.0, 0.0, 0.0, 0.0};
  if (i0 < n) {
    const int n0 = a.pa.grid.n[0], n1 = a.pa.grid.n[1], n2 = a.pa.grid.n[2];
    const uint32_t sxi = valid ? S.sx[i] : 0u, syi = valid ? S.sy[i] : 0u,
                   szi = valid ? S.sz[i] : 0u;
    real qi = (real)0;
    if (COUL && valid) qi = sizeof(real) == 8 ? (real)S.qd[i] : (real)S.qf[i];
    const int ti = (MULTI && valid) ? S.type[i] : 0;
    const uint32_t idi = valid ? (uint32_t)a.id[i] : 0u;
    const int cx = cell_of(sxi, n0), cy = cell_of(syi, n1), cz = cell_of(szi, n2);
    int ncore = 0, nsh = 0, cnt = 0;
    auto flush = [&]() {
      const int maxc = __reduce_max_sync(FULL, cnt);
      for (int t = 0; t < maxc; ++t)
        if (t < cnt) rbl_pair<real, COUL, MULTI>(a, tab, sxi, syi, szi, qi, ti, list[wid][t][lane], core);
      cnt = 0;
      __syncwarp();
    };
    unsigned remaining = __ballot_sync(FULL, valid);
    while (remaining) {
      const int leader = __ffs(remaining) - 1;
      const int gx = __shfl_sync(FULL, cx, leader), gy = __shfl_sync(FULL, cy, leader),
                gz = __shfl_sync(FULL, cz, leader);
      const bool in = valid && cx == gx && cy == gy && cz == gz;
      remaining &= ~__ballot_sync(FULL, in);
      const uint32_t ox = __shfl_sync(FULL, sxi, leader), oy = __shfl_sync(FULL, syi, leader),
                     oz = __shfl_sync(FULL, szi, leader);
      const float xi = (float)(int)(sxi - ox) * a.pa.pc.h[0];
      const float yi = (float)(int)(syi - oy) * a.pa.pc.h[1];
      const float zi = (float)(int)(szi - oz) * a.pa.pc.h[2];
      // draws of pass 2, kept sorted by index (stable in t)
      uint32_t idx[kRblMaxP];
      int ord[kRblMaxP];
      int ndraw = 0;
      for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
          flush();
          if (in) {
            for (int t = 0; t < a.p; ++t)
              if (a.partners) a.partners[i * a.p + t] = -1;
            if (nsh > a.p) {
              const uint32_t st = (uint32_t)(*a.step);
              for (int t = 0; t < a.p; t += 4) {
                const uint4 w = philox4x32_10(make_uint4(idi, (uint32_t)(t / 4), st, 1u), a.key);
                const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
                for (int u = 0; u < 4 && t + u < a.p; ++u)
                  idx[t + u] = (uint32_t)(((uint64_t)ww[u] * (uint64_t)nsh) >> 32);
              }
              ndraw = a.p;
              for (int t = 0; t < ndraw; ++t) ord[t] = t;
              for (int t = 1; t < ndraw; ++t) {  // insertion sort by idx, stable
                const int v = ord[t];
                int u = t - 1;
                while (u >= 0 && idx[ord[u]] > idx[v]) { ord[u + 1] = ord[u]; --u; }
                ord[u + 1] = v;
              }
            }
          }
        }
        int kshell = 0, ptr = 0;
        for (int dz = -1; dz <= 1; ++dz) {
          const int rz = ((gz + dz) % n2 + n2) % n2;
          for (int dy = -1; dy <= 1; ++dy) {
            const int ry = ((gy + dy) % n1 + n1) % n1;
            for (int dx = -1; dx <= 1; ++dx) {
              const int rx = ((gx + dx) % n0 + n0) % n0;
              const int64_t cell = rx + (int64_t)n0 * (ry + (int64_t)n1 * rz);
              const int64_t j0 = S.cell_start[cell], j1 = S.cell_start[cell + 1];
              for (int64_t base = j0; base < j1; base += 32) {
                if (pass == 0 && __any_sync(FULL, cnt > kListK - 32)) flush();
                const int64_t jj = base + lane;
                if (jj < j1)
                  stage[wid][lane] = make_float4((float)(int)(S.sx[jj] - ox) * a.pa.pc.h[0],
                                                 (float)(int)(S.sy[jj] - oy) * a.pa.pc.h[1],
                                                 (float)(int)(S.sz[jj] - oz) * a.pa.pc.h[2], 0.f);
                __syncwarp();
                const int nj = (int)min((int64_t)32, j1 - base);
                for (int t = 0; t < nj; ++t) {
                  const float4 pj = stage[wid][t];
                  float ddx = xi - pj.x, ddy = yi - pj.y, ddz = zi - pj.z;
                  if (WRAP) {
                    ddx = fold(ddx, a.pa.L[0], a.pa.invL[0]);
                    ddy = fold(ddy, a.pa.L[1], a.pa.invL[1]);
                    ddz = fold(ddz, a.pa.L[2], a.pa.invL[2]);
                  }
                  const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                  const int64_t j = base + t;
                  const int cls = (in && j != i && r2 <= a.rs2_hi) ? rbl_classify(a, r2, sxi, syi, szi, j) : 0;
                  if (pass == 0) {
                    list[wid][cnt][lane] = (int32_t)j;
                    cnt += cls == 1 ? 1 : 0;
                    ncore += cls == 1 ? 1 : 0;
                    nsh += cls == 2 ? 1 : 0;
                  } else if (cls == 2) {
                    if (nsh <= a.p) {
                      rbl_pair<real, COUL, MULTI>(a, tab, sxi, syi, szi, qi, ti, j, shell);
                      if (a.partners) a.partners[i * a.p + kshell] = a.id[j];
                    } else {
                      while (ptr < ndraw && idx[ord[ptr]] == (uint32_t)kshell) {
                        rbl_pair<real, COUL, MULTI>(a, tab, sxi, syi, szi, qi, ti, j, shell);
                        if (a.partners) a.partners[i * a.p + ord[ptr]] = a.id[j];
                        ++ptr;
                      }
                    }
                    ++kshell;
                  }
                }
                __syncwarp();
              }
            }
          }
        }
      }
    }
    if (valid) {
      const real w = nsh > a.p ? (real)nsh / (real)a.p : (real)1;
      fx = core.fx + w * shell.fx;
      fy = core.fy + w * shell.fy;
      fz = core.fz + w * shell.fz;
      en[Q_UREAL] = ((double)core.uc - (double)core.cuc) +
                    (double)w * ((double)shell.uc - (double)shell.cuc);
      en[Q_ULJ] = (double)(core.ulj + w * shell.ulj);
      en[Q_WREAL] = ((double)core.wc - (double)core.cwc) +
                    (double)w * ((double)shell.wc - (double)shell.cwc);
      en[Q_WLJ] = (double)(core.wlj + w * shell.wlj);
      const int64_t St = a.pa.Fstride;
      if (sizeof(real) == 8) { a.pa.Fd[i] = (double)fx; a.pa.Fd[St + i] = (double)fy; a.pa.Fd[2 * St + i] = (double)fz; }
      else { a.pa.F[i] = (float)fx; a.pa.F[St + i] = (float)fy; a.pa.F[2 * St + i] = (float)fz; }
      if (a.ncore) a.ncore[i] = ncore;
      if (a.nshell) a.nshell[i] = nsh;
    }
  }
  double v[NQ_PAIR + 3] = {en[0], en[1], en[2], en[3], (double)fx, (double)fy, (double)fz};
#pragma unroll
  for (int k = 0; k < NQ_PAIR + 3; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) wred[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < NQ_PAIR + 3) {
    double s = 0.0;
    for (int w = 0; w < kRblWarps; ++w) s += wred[w][threadIdx.x];
    if (threadIdx.x < NQ_PAIR) a.pa.epart[(int64_t)blockIdx.x * NQ_PAIR + threadIdx.x] = 0.5 * s;
    else a.fsum_part[(int64_t)blockIdx.x * 3 + threadIdx.x - NQ_PAIR] = s;
  }
}

// Mean of F~ over all particles (fixed-order FP64), then F -= mean (Eq. F_corr).
__global__ void __launch_bounds__(256) rbl_mean_kernel(const double *__restrict__ part, int64_t nblk,
                                                       int64_t N, double *__restrict__ mean) {
  __shared__ double sh[3][256];
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b * 3 + k];
    sh[k][threadIdx.x] = s;
  }
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 3) mean[threadIdx.x] = sh[threadIdx.x][0] / (double)N;
}

template <typename real>
__global__ void rbl_subtract_kernel(real *__restrict__ F, int64_t N, const double *__restrict__ mean) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  F[i] -= (real)mean[0];
  F[N + i] -= (real)mean[1];
  F[2 * N + i] -= (real)mean[2];
}

int64_t rbl_blocks(int64_t n) { return (n + 32 * kRblWarps - 1) / (32 * kRblWarps); }

template <typename real, bool COUL>
static void rbl_launch(const RblArgs &a, int64_t blocks, bool multi, bool wrap, cudaStream_t st) {
  const dim3 g((unsigned)blocks), b(kRblWarps * 32);
  if (wrap) {
    if (multi) rbl_kernel<real, COUL, true, true><<<g, b, 0, st>>>(a);
    else rbl_kernel<real, COUL, false, true><<<g, b, 0, st>>>(a);
  } else {
    if (multi) rbl_kernel<real, COUL, true, false><<<g, b, 0, st>>>(a);
    else rbl_kernel<real, COUL, false, false><<<g, b, 0, st>>>(a);
  }
}

cudaError_t launch_rbl(Ctx &c, bool want_debug) {
  const int b = c.cur;
  RblArgs a;
  PairArgs &pa = a.pa;
  pa.grid = c.grid;
  pa.pc = c.pc;
  pa.eps24 = c.lj.eps24[0]; pa.eps4 = c.lj.eps4[0]; pa.sig2 = c.lj.sig2[0];
  pa.eps24d = c.lj.eps24d[0]; pa.eps4d = c.lj.eps4d[0]; pa.sig2d = c.lj.sig2d[0];
  pa.table = reinterpret_cast<const LJTable *>(c.lj_dev);
  pa.F = c.F; pa.Fd = c.Fd; pa.Fstride = c.N; pa.accumulate = 0;
  pa.set.sx = c.s[b]; pa.set.sy = c.s[b] + c.N; pa.set.sz = c.s[b] + 2 * c.N;
  pa.set.qf = c.qf[b]; pa.set.qd = c.qd[b]; pa.set.type = c.type[b];
  pa.set.cell_start = c.cell_start; pa.set.map = nullptr; pa.set.n = c.N;
  pa.epart = c.epart + c.off_rbl;
  pa.nbr = nullptr;
  a.id = c.id[b];
  const double rc2 = c.rc * c.rc, rk2 = c.r_core * c.r_core;
  a.rcore2_lo = (float)(rk2 * (1.0 - 1e-5)); a.rcore2_hi = (float)(rk2 * (1.0 + 1e-5));
  a.rs2_lo = (float)(rc2 * (1.0 - 1e-5)); a.rs2_hi = (float)(rc2 * (1.0 + 1e-5));
  a.rcore2d = rk2; a.rs2d = rc2;
  a.p = c.p_rbl;
  a.key = make_uint2((uint32_t)c.seed, (uint32_t)(c.seed >> 32) ^ c.replica);
  a.step = c.step_dev;
  a.fsum_part = c.rbl_part;
  a.ncore = want_debug ? c.nbr : nullptr;
  a.nshell = want_debug ? c.nshell : nullptr;
  a.partners = want_debug ? c.partners : nullptr;
  const int64_t blocks = rbl_blocks(c.N);
  const bool multi = c.nt > 1, coul = c.Nq > 0;
  // groups share one cell: the leader frame is a valid minimum image while a + r_s < L/2
  bool wrap = false;
  for (int d = 0; d < 3; ++d) {
    pa.L[d] = (float)c.box[d];
    pa.invL[d] = (float)(1.0 / c.box[d]);
    if (!(c.box[d] / c.grid.n[d] + c.rc < 0.5 * c.box[d] * (1.0 - 1e-9))) wrap = true;
  }
  pa.smax = 1;
  pa.comp = c.precision == RBE_FP32_COMP;
  if (c.precision == RBE_FP64) {
    if (coul) rbl_launch<double, true>(a, blocks, multi, wrap, c.stream);
    else rbl_launch<double, false>(a, blocks, multi, wrap, c.stream);
  } else {
    if (coul) rbl_launch<float, true>(a, blocks, multi, wrap, c.stream);
    else rbl_launch<float, false>(a, blocks, multi, wrap, c.stream);
  }
  mark(c, RBE_PH_PAIR2);
  rbl_mean_kernel<<<1, 256, 0, c.stream>>>(c.rbl_part, blocks, c.N, c.rbl_mean);
  const unsigned nb = (unsigned)((c.N + 255) / 256);
  if (c.precision == RBE_FP64) rbl_subtract_kernel<double><<<nb, 256, 0, c.stream>>>(c.Fd, c.N, c.rbl_mean);
  else rbl_subtract_kernel<float><<<nb, 256, 0, c.stream>>>(c.F, c.N, c.rbl_mean);
  return cudaGetLastError();
}

}  // namespace rbe
