// k_cpair.cu -- real-space pair forces over clusters of particles, each pair evaluated once
// (Newton's third law), for the cell-list real space (Eqs. F_i, G_short, LJ):
//
//   F_i += sum_{j != i, r_ij <= r_c} (C q_i q_j G(r) + G_LJ(r)) (r_i - r_j),   F_j -= the same.
//
// Clusters. Particles are sorted by (cell, s_x, id) with cells of r_c / sub, so each row of
// cells (c_y, c_z) holds its particles in ascending s_x. A cluster is 8 consecutive
// particles of a row (the last cluster of a row may hold fewer) and a super-cluster is up
// to NC consecutive clusters of a row: one warp's work. Global cluster indices run over the
// rows in order (cl_base per row), and so do the super-clusters (sc_base per row).
//
// Half list. The cluster pair (I, J) is evaluated once, by the super-cluster that holds I,
// when I <= J (global index) and the bounding boxes of I and J are within r_c of each
// other. Every particle pair within r_c lies in one such pair of clusters, or inside one
// cluster (I = J: then only particle a with particle b > a of the cluster).
//
// Lanes. Lane (h, a) = (lane / 8, lane % 8) holds particle a of every i-cluster of the
// super-cluster (coordinates and force in registers) and particles h and h + 4 of the
// j-cluster being visited, so one visit evaluates the 8 x 8 pairs of every i-cluster the
// visit's mask names, two per lane. The reaction on j is summed over the 8 lanes that
// share h by shuffles, once per visit, and added to j's force.
//
// Forces are summed in 64-bit fixed point by integer atomics. Integer sums do not depend on
// their order, so the forces are the same run to run; a final pass converts them to
// floating point. Energies and virials are per-block partial sums, as in the other kernels.
//
// Frame. A super-cluster's coordinates are the exact integer offsets of its particles from
// the centre of its bounding box, converted to FP32 (kept as integers in the FP64 form). A
// visited j particle's x is converted the same way; its y and z are the frame coordinates of
// its cluster's box corner plus its FP32 offsets from that corner, stored per step in the
// cluster's eight record slots (a cluster lies in one cell in y and z, so the offsets are
// small and never wrap; the one extra rounding widens the band below).
// The difference of two offsets is the minimum-image displacement of a pair within r_c as
// long as the super-cluster's extent plus 2 r_c stays below L on every axis: the host
// checks y and z (a cell width), the kernel splits a super-cluster whose x extent is
// larger into groups of clusters that fit, down to single particles. The cutoff decision is exact: FP32 outside a
// band around r_c^2 that covers the rounding of the frame coordinates, and the oracle's
// FP64 expression of the integer displacement inside it (a rare branch per visit whose
// pairs are added by atomics); the FP64 form always takes the FP64 expression.
#include <climits>
#include <cmath>

#include "pair_common.cuh"

namespace rbe {

constexpr int kClSize = 8;              // particles per cluster
constexpr int kCpMaxRows = 49;          // (2R+1)^2 stencil rows for R <= 3
constexpr int kCpMaxSeg = 2 * kCpMaxRows;

struct ClusterArgs {
  PairSet set;                 // full sorted set
  Grid grid;
  PairConst pc;
  float ljA, ljB, ljA12, ljB6;
  double ljAd, ljBd, ljA12d, ljB6d;
  const LJTable *table;        // device copy, multi-type only
  const int32_t *cl_base;      // nrows + 1: first global cluster of each row
  const int32_t *sc_base;      // nrows + 1: first super-cluster of each row
  const uint4 *cl_lo, *cl_hi;  // per cluster: (min s_x, s_y, s_z, first particle), (max..., count)
  const uint4 *jrec;           // FP32 forms: 8 slots per cluster (s_x, y and z offsets from the
                               // box corner as FP32 bits, q bits); empty slots y = -3e18
  int nrows;
  long long *facc;             // 3 x N fixed-point forces (x block, y, z)
  int64_t N;
  float fscale;                // fixed-point scale (FP32 forms)
  double fscale_d;             // (FP64 form)
  double *epart;               // per-block partials (NQ_PAIR doubles)
  int32_t *nbr;                // neighbour counts (sorted order, zeroed before), nullable
  int comp;                    // Kahan sums for the Coulomb energy and virial
  uint32_t xlim;               // largest x extent of a cluster group the frame allows
  float bb2;                   // bounding-box test: squared gap <= bb2 (r_c^2, widened)
  float rc2_mid, rc2_half;     // band test: |r^2 - rc2_mid| <= rc2_half covers [rc2_lo, rc2_hi]
  int *err;
  int64_t nslots;              // the pass's energy partial slots (at least the grid)
};

// ---------------------------------------------------------------------------------------
// Per-step cluster tables

struct RowsArgs {
  const int32_t *cell_start;
  int n0, nrows, nc_sc;
  int32_t *cl_base, *sc_base;
};
struct BoundsArgs {
  const uint32_t *sx, *sy, *sz;
  const float *qf;
  const int32_t *cell_start;
  int n0, nrows;
  const int32_t *cl_base;
  int64_t cap;
  uint4 *lo, *hi;
  uint4 *jrec;                 // nullable (FP64 form)
  float hy, hz;                // length of one fractional unit in y and z
};
struct FinishArgs {
  long long *facc;
  void *F;                 // float or double forces, by the kernel's type
  int64_t n3;
  float sh, sl;
  double inv_scale;
};

// One block: clusters and super-clusters of every row, as exclusive prefix sums.
__device__ __forceinline__ void cluster_rows_body(const RowsArgs &a, int, int) {
  __shared__ int2 ws[32];
  const int32_t *__restrict__ cell_start = a.cell_start;
  const int n0 = a.n0, nrows = a.nrows, nc_sc = a.nc_sc;
  int32_t *__restrict__ cl_base = a.cl_base;
  int32_t *__restrict__ sc_base = a.sc_base;
  const unsigned FULL = 0xffffffffu;
  const int t = threadIdx.x, ln = t & 31;
  const int per = (nrows + 1023) / 1024;
  const int r0 = min(nrows, t * per), r1 = min(nrows, r0 + per);
  int cl = 0, sc = 0;
  for (int r = r0; r < r1; ++r) {
    const int n = cell_start[(int64_t)(r + 1) * n0] - cell_start[(int64_t)r * n0];
    const int k = (n + kClSize - 1) / kClSize;
    cl += k;
    sc += (k + nc_sc - 1) / nc_sc;
  }
  int icl = cl, isc = sc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(FULL, icl, o), v = __shfl_up_sync(FULL, isc, o);
    if (ln >= o) { icl += u; isc += v; }
  }
  if (ln == 31) ws[t >> 5] = make_int2(icl, isc);
  __syncthreads();
  if (t < 32) {
    const int2 v = ws[t];
    int u = v.x, w = v.y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int p = __shfl_up_sync(FULL, u, o), q = __shfl_up_sync(FULL, w, o);
      if (ln >= o) { u += p; w += q; }
    }
    ws[t] = make_int2(u - v.x, w - v.y);
  }
  __syncthreads();
  int bc = ws[t >> 5].x + icl - cl, bs = ws[t >> 5].y + isc - sc;
  for (int r = r0; r < r1; ++r) {
    const int n = cell_start[(int64_t)(r + 1) * n0] - cell_start[(int64_t)r * n0];
    const int k = (n + kClSize - 1) / kClSize;
    cl_base[r] = bc;
    sc_base[r] = bs;
    bc += k;
    bs += (k + nc_sc - 1) / nc_sc;
  }
  if (t == 1023) {
    cl_base[nrows] = bc;
    sc_base[nrows] = bs;
  }
}
RBE_BATCHED_KERNEL(__launch_bounds__(1024), cluster_rows_kernel, RowsArgs, cluster_rows_body)

// Largest r in [0, nrows) with base[r] <= g (base is non-decreasing; g < base[nrows]).
__device__ __forceinline__ int row_of(const int32_t *__restrict__ base, int nrows, int g) {
  int lo = 0, hi = nrows - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Bounding box (integer fractional coordinates), first particle and count of every cluster,
// and its j records: slot k holds particle k's s_x, its y and z offsets from the box's low
// corner in length units (FP32 bits) and its charge bits; a slot past the cluster's count
// holds y = -3e18, beyond the reach of any i particle. Eight threads per cluster, one per
// slot, with the box reduced over the eight by shuffles.
static_assert(kClSize == 8, "eight threads per cluster");
__device__ __forceinline__ void cluster_bounds_body(const BoundsArgs &a, int bx, int) {
  const int32_t *__restrict__ cell_start = a.cell_start;
  const int32_t *__restrict__ cl_base = a.cl_base;
  const int n0 = a.n0, nrows = a.nrows;
  const int64_t t = (int64_t)bx * blockDim.x + threadIdx.x;
  const int64_t g = t >> 3;
  const int k = (int)(t & 7);
  // (the same for the eight threads of a cluster, which exit together)
  if (g >= a.cap || g >= cl_base[nrows]) return;
  const unsigned gm = 0xffu << (threadIdx.x & 24);
  const int r = row_of(cl_base, nrows, (int)g);
  const int ps = cell_start[(int64_t)r * n0], pe = cell_start[(int64_t)(r + 1) * n0];
  const int b = ps + (int)(g - cl_base[r]) * kClSize;
  const int n = min(kClSize, pe - b);
  const bool v = k < n;
  uint32_t x = 0u, y = 0u, z = 0u;
  float q = 0.f;
  if (v) {
    x = a.sx[b + k]; y = a.sy[b + k]; z = a.sz[b + k];
    q = a.qf[b + k];
  }
  uint32_t x0 = v ? x : 0xffffffffu, y0 = v ? y : 0xffffffffu, z0 = v ? z : 0xffffffffu;
  uint32_t x1 = x, y1 = y, z1 = z;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    x0 = min(x0, __shfl_xor_sync(gm, x0, o)); x1 = max(x1, __shfl_xor_sync(gm, x1, o));
    y0 = min(y0, __shfl_xor_sync(gm, y0, o)); y1 = max(y1, __shfl_xor_sync(gm, y1, o));
    z0 = min(z0, __shfl_xor_sync(gm, z0, o)); z1 = max(z1, __shfl_xor_sync(gm, z1, o));
  }
  if (k == 0) {
    a.lo[g] = make_uint4(x0, y0, z0, (uint32_t)b);
    a.hi[g] = make_uint4(x1, y1, z1, (uint32_t)n);
  }
  if (a.jrec)
    a.jrec[t] = v ? make_uint4(x, __float_as_uint((float)(int)(y - y0) * a.hy),
                               __float_as_uint((float)(int)(z - z0) * a.hz), __float_as_uint(q))
                  : make_uint4(0u, __float_as_uint(-3e18f), 0u, 0u);
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), cluster_bounds_kernel, BoundsArgs, cluster_bounds_body)

// F = fixed-point sums / scale (overwriting), and the sums cleared for the next pass. The
// 64-bit sum converts as its two 32-bit halves (a 64-bit integer conversion is slow here):
// v = hi 2^32 + lo with hi signed and lo unsigned; FP32 forms take the FP32 factors
// sh = 2^32 / scale and sl = 1 / scale (no FP64 work per element), the FP64 form the FP64 ones.
// Four sums a thread in 16-byte accesses (one 8-byte sum a thread left most of the pass
// waiting on memory latency).
template <typename real>
__device__ __forceinline__ real fx_value(long long v, const FinishArgs &a) {
  const int hi = (int)(v >> 32);
  const unsigned lo = (unsigned)(v & 0xffffffffll);
  if (sizeof(real) == 8) return (real)(((double)hi * 4294967296.0 + (double)lo) * a.inv_scale);
  return (real)fmaf((float)hi, a.sh, (float)lo * a.sl);
}

template <typename real>
__device__ __forceinline__ void cpair_finalize_body(const FinishArgs &a, int bx, int) {
  const int64_t k0 = 4 * ((int64_t)bx * blockDim.x + threadIdx.x);
  const int64_t n3 = a.n3;
  if (k0 >= n3) return;
  long long *__restrict__ facc = a.facc;
  real *__restrict__ F = static_cast<real *>(a.F);
  if (k0 + 4 <= n3) {  // facc and F start 256-byte aligned, k0 is a multiple of 4
    const longlong2 u = *reinterpret_cast<const longlong2 *>(facc + k0);
    const longlong2 w = *reinterpret_cast<const longlong2 *>(facc + k0 + 2);
    *reinterpret_cast<longlong2 *>(facc + k0) = make_longlong2(0, 0);
    *reinterpret_cast<longlong2 *>(facc + k0 + 2) = make_longlong2(0, 0);
    const real f0 = fx_value<real>(u.x, a), f1 = fx_value<real>(u.y, a);
    const real f2 = fx_value<real>(w.x, a), f3 = fx_value<real>(w.y, a);
    if (sizeof(real) == 4) {
      *reinterpret_cast<float4 *>(F + k0) = make_float4((float)f0, (float)f1, (float)f2, (float)f3);
    } else {
      *reinterpret_cast<double2 *>(F + k0) = make_double2((double)f0, (double)f1);
      *reinterpret_cast<double2 *>(F + k0 + 2) = make_double2((double)f2, (double)f3);
    }
  } else {
    for (int64_t k = k0; k < n3; ++k) {
      const long long v = facc[k];
      facc[k] = 0;
      F[k] = fx_value<real>(v, a);
    }
  }
}
template <typename real>
__global__ void __launch_bounds__(256) cpair_finalize_kernel(const FinishArgs a) {
  cpair_finalize_body<real>(a, (int)blockIdx.x, (int)gridDim.x);
}
template <typename real>
__global__ void __launch_bounds__(256)
    cpair_finalize_kernel_b(const FinishArgs *__restrict__ t, const int32_t *__restrict__ pre,
                            int nrep) {
  const BatchIdx q = batch_locate(pre, nrep);
  cpair_finalize_body<real>(t[q.r], q.bx, q.nbx);
}

// ---------------------------------------------------------------------------------------
// Pair evaluation

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <typename real>
struct CpAcc {
  real u0, u1;   // single type: sum r^-12, sum r^-6; several types: U_LJ, W_LJ
  real uc, wc, cuc, cwc;  // Coulomb energy and virial (Kahan compensations)
};

// LJ and Coulomb terms of one pair at squared distance r2 inside the cutoff (1/r^2 = 0 and
// qq = 0 give exact zeros); returns the force factor g (F_i += g (r_i - r_j)).
template <typename real, bool COUL, bool MULTI>
__device__ __forceinline__ real cp_terms(const ClusterArgs &a, bool in, real r2, real ir2,
                                         real qi, real qj, int ti, int tj, CpAcc<real> &acc) {
  real g;
  const real ir6 = ir2 * ir2 * ir2;
  if (MULTI) {
    const LJTable *tab = a.table;
    const int pt = ti * tab->nt + tj;
    real A, B, A12, B6;
    if (sizeof(real) == 8) { A = (real)tab->Ad[pt]; B = (real)tab->Bd[pt]; A12 = (real)tab->A12d[pt]; B6 = (real)tab->B6d[pt]; }
    else { A = (real)tab->A[pt]; B = (real)tab->B[pt]; A12 = (real)tab->A12[pt]; B6 = (real)tab->B6[pt]; }
    const real w = ir6 * mad(A12, ir6, -B6);
    g = w * ir2;
    acc.u0 = mad(ir6, mad(A, ir6, -B), acc.u0);
    acc.u1 += w;
  } else {
    const real A12 = sizeof(real) == 8 ? (real)a.ljA12d : (real)a.ljA12;
    const real B6 = sizeof(real) == 8 ? (real)a.ljB6d : (real)a.ljB6;
    g = ir6 * ir2 * mad(A12, ir6, -B6);
    acc.u0 = mad(ir6, ir6, acc.u0);
    acc.u1 += ir6;
  }
  if (COUL) {
    const real qq = qi * qj;
    if (in && qq != (real)0) {
      const PairConst &pc = a.pc;
      real r, rinv, erfcv, expv;
      if (sizeof(real) == 8) {
        r = (real)sqrt((double)r2);
        rinv = (real)1 / r;
        erfcv = (real)erfc(pc.sqrt_alpha_d * (double)r);
        expv = (real)exp(-pc.alpha_d * (double)r2);
      } else {
        rinv = (real)rsqrtf((float)r2);
        r = r2 * rinv;
        erfcv = (real)erfcf(pc.sqrt_alpha * (float)r);
        expv = (real)expf(-pc.alpha * (float)r2);
      }
      const real Cqq = (sizeof(real) == 8 ? (real)pc.C_d : (real)pc.C) * qq;
      const real tsp = sizeof(real) == 8 ? (real)pc.two_sqrt_alpha_over_sqrt_pi_d
                                         : (real)pc.two_sqrt_alpha_over_sqrt_pi;
      const real rinv2 = rinv * rinv;
      const real gc = Cqq * mad(erfcv * rinv, rinv2, tsp * expv * rinv2);
      g += gc;
      if (a.comp) {
        kahan_add(acc.uc, acc.cuc, Cqq * erfcv * rinv);
        kahan_add(acc.wc, acc.cwc, gc * r2);
      } else {
        acc.uc = mad(Cqq * erfcv, rinv, acc.uc);
        acc.wc = mad(gc, r2, acc.wc);
      }
    }
  }
  return g;
}

// ---------------------------------------------------------------------------------------
// The kernel: one warp per super-cluster.

template <typename real, bool COUL, bool MULTI, bool COUNT>
__device__ __forceinline__ void cpair_body(const ClusterArgs &a, int bx, int nbx) {
  constexpr bool F64 = sizeof(real) == 8;
  constexpr int NC = F64 ? 4 : 8;          // clusters per super-cluster
  constexpr int NP = NC * kClSize;         // particles per super-cluster
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ uint4 si[NP];                 // s_x, s_y, s_z, charge bits
  __shared__ int32_t sti[MULTI ? NP : 1];
  __shared__ float4 ibl[NC], ibh[NC];      // i-cluster boxes in frame coordinates
  // FP32 forms: the group's i particles in frame coordinates (x, y, z, charge), read once
  // per i-cluster and visit; slots outside the group hold a point no j can reach
  __shared__ float4 sif[F64 ? 1 : NP];
  __shared__ int32_t seg_beg[kCpMaxSeg], seg_pre[kCpMaxSeg + 1];
  const int lane = threadIdx.x, a8 = lane & 7, hh = lane >> 3;
  const int w = bx;
  const PairConst &pc = a.pc;
  const int64_t N = a.N;
  CpAcc<real> acc;
  acc.u0 = acc.u1 = acc.uc = acc.wc = acc.cuc = acc.cwc = (real)0;
  const int nrows = a.nrows;
  if (w < a.sc_base[nrows]) {
    const int r = row_of(a.sc_base, nrows, w);
    const int n0 = a.grid.n[0], n1 = a.grid.n[1], n2 = a.grid.n[2];
    const int ps = a.set.cell_start[(int64_t)r * n0], pe = a.set.cell_start[(int64_t)(r + 1) * n0];
    const int ksc = w - a.sc_base[r];
    const int g0 = a.cl_base[r] + ksc * NC;
    const int nc = min(NC, a.cl_base[r + 1] - a.cl_base[r] - ksc * NC);
    const int p0 = ps + ksc * NP;
    const int np = min(NP, pe - p0);
    const int cy = r % n1, cz = r / n1;
    // (slots past the particles hold type 0 and no charge: masked lanes still look up the
    // LJ table by type before their result is zeroed)
    for (int t = lane; t < NP; t += 32) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      int ty = 0;
      if (t < np) {
        const int p = p0 + t;
        v = make_uint4(a.set.sx[p], a.set.sy[p], a.set.sz[p],
                       COUL ? __float_as_uint(a.set.qf[p]) : 0u);
        if (MULTI) ty = a.set.type[p];
      }
      si[t] = v;
      if (MULTI) sti[t] = ty;
    }
    __syncwarp();
    // Groups of consecutive clusters whose x extent the frame allows (normally one group).
    // A single cluster wider than that is taken one particle at a time (asub), as a group
    // of one point.
    int cb = 0, asub = -1;
    while (cb < nc) {
      int ce = cb + 1;
      if (asub < 0) {
        const uint32_t xfirst = si[kClSize * cb].x;
        while (ce < nc && si[min(np, kClSize * (ce + 1)) - 1].x - xfirst <= a.xlim) ++ce;
        if (si[min(np, kClSize * ce) - 1].x - xfirst > a.xlim) asub = 0;
      }
      const int q0 = asub < 0 ? kClSize * cb : kClSize * cb + asub;
      const int q1 = asub < 0 ? min(np, kClSize * ce) : q0 + 1;
      // group box and frame centre (no wrap inside a row: x ascending, y and z in one cell)
      uint32_t ylo = 0xffffffffu, yhi = 0u, zlo = 0xffffffffu, zhi = 0u;
      for (int t = q0 + lane; t < q1; t += 32) {
        const uint4 v = si[t];
        ylo = min(ylo, v.y); yhi = max(yhi, v.y);
        zlo = min(zlo, v.z); zhi = max(zhi, v.z);
      }
      ylo = __reduce_min_sync(FULL, ylo); yhi = __reduce_max_sync(FULL, yhi);
      zlo = __reduce_min_sync(FULL, zlo); zhi = __reduce_max_sync(FULL, zhi);
      const uint32_t xlo = si[q0].x, xhi = si[q1 - 1].x;
      const uint32_t rx = xlo + ((xhi - xlo) >> 1), ry = ylo + ((yhi - ylo) >> 1),
                     rz = zlo + ((zhi - zlo) >> 1);
      // i particles of this lane: particle a8 of each cluster of the group
      real fxi[NC], fyi[NC], fzi[NC], qi[NC];
      int oxi[NC], oyi[NC], ozi[NC], ti[NC], cnti[NC];
      bool vi[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int t = kClSize * c + a8;
        const bool v = c >= cb && c < ce && t < np && (asub < 0 || a8 == asub);
        vi[c] = v;
        const uint4 s = si[t];
        oxi[c] = (int)(s.x - rx); oyi[c] = (int)(s.y - ry); ozi[c] = (int)(s.z - rz);
        qi[c] = COUL ? (real)__uint_as_float(s.w) : (real)0;
        if (COUL && F64 && v) qi[c] = (real)a.set.qd[p0 + t];
        ti[c] = MULTI ? sti[t] : 0;
        fxi[c] = fyi[c] = fzi[c] = (real)0;
        cnti[c] = 0;
      }
      if (!F64) {
        for (int t = lane; t < NP; t += 32) {
          const int c = t / kClSize, a_ = t % kClSize;
          const bool v = c >= cb && c < ce && t < np && (asub < 0 || a_ == asub);
          const uint4 s = si[t];
          sif[t] = v ? make_float4((float)(int)(s.x - rx) * pc.h[0], (float)(int)(s.y - ry) * pc.h[1],
                                   (float)(int)(s.z - rz) * pc.h[2], __uint_as_float(s.w))
                     : make_float4(3e18f, 3e18f, 3e18f, 0.f);
        }
      }
      // i-cluster boxes in the frame (lanes cb..ce-1)
      if (lane < NC) {
        float4 lo4 = make_float4(3e18f, 3e18f, 3e18f, 0.f), hi4 = make_float4(3e18f, 3e18f, 3e18f, 0.f);
        if (lane >= cb && lane < ce) {
          uint4 l, u;
          if (asub < 0) { l = a.cl_lo[g0 + lane]; u = a.cl_hi[g0 + lane]; }
          else { l = u = si[q0]; }  // the one particle of a point group
          lo4 = make_float4((float)(int)(l.x - rx) * pc.h[0], (float)(int)(l.y - ry) * pc.h[1],
                            (float)(int)(l.z - rz) * pc.h[2], 0.f);
          hi4 = make_float4((float)(int)(u.x - rx) * pc.h[0], (float)(int)(u.y - ry) * pc.h[1],
                            (float)(int)(u.z - rz) * pc.h[2], 0.f);
        }
        ibl[lane] = lo4;
        ibh[lane] = hi4;
      }
      // Candidate j-clusters: for each stencil row (dy, dz), the clusters holding the row's
      // particles within the group's x-reach (one lane per row; a row wraps into at most
      // two parts), from the group's first global cluster on; a warp scan gives offsets.
      const int R1 = a.grid.R[1], R2 = a.grid.R[2];
      const int ny = 2 * R1 + 1, nrst = ny * (2 * R2 + 1);
      const int gxlo = (int)(xlo - rx), gxhi = (int)(xhi - rx);
      const int gylo = (int)(ylo - ry), gyhi = (int)(yhi - ry);
      const int gzlo = (int)(zlo - rz), gzhi = (int)(zhi - rz);
      const int jmin = g0 + cb;
      int carry = 0;
      for (int rb = 0; rb < nrst; rb += 32) {
        const int t = rb + lane;
        int b0 = 0, l0 = 0, b1 = 0, l1 = 0;
        if (t < nrst) {
          const int dz = t / ny - R2, dy = t % ny - R1;
          const int ryw = ((cy + dy) % n1 + n1) % n1, rzw = ((cz + dz) % n2 + n2) % n2;
          const int r2i = ryw + n1 * rzw;
          const int qs = a.set.cell_start[(int64_t)r2i * n0];
          const int qe = a.set.cell_start[(int64_t)(r2i + 1) * n0];
          if (qe > qs) {
            // the row's y and z extent in frame units (unwrapped, widened by 2 units), its
            // distance from the group's box, and the x-reach that is left
            const int64_t W32 = (int64_t)1 << 32;
            const int64_t y0 = (int64_t)(cy + dy) * W32 / n1 - (int64_t)ry - 2;
            const int64_t y1 = (int64_t)(cy + dy + 1) * W32 / n1 - (int64_t)ry + 2;
            const int64_t z0 = (int64_t)(cz + dz) * W32 / n2 - (int64_t)rz - 2;
            const int64_t z1 = (int64_t)(cz + dz + 1) * W32 / n2 - (int64_t)rz + 2;
            const int64_t ey = max((int64_t)0, max(y0 - gyhi, (int64_t)gylo - y1));
            const int64_t ez = max((int64_t)0, max(z0 - gzhi, (int64_t)gzlo - z1));
            const float dyl = (float)ey * pc.h[1], dzl = (float)ez * pc.h[2];
            const float rx2 = a.bb2 - dyl * dyl - dzl * dzl;
            if (rx2 > 0.f) {
              const int64_t reach = (int64_t)(sqrtf(rx2) * (1.0f + 1e-5f) / pc.h[0]) + 4;
              const int64_t X0 = (int64_t)rx + gxlo - reach, X1 = (int64_t)rx + gxhi + reach;
              const int64_t W = (int64_t)1 << 32;
              // first particle of [qs, qe) with s_x >= key (rows are sorted by s_x)
              auto first_ge = [&](int64_t key) {
                int lo = qs, hi = qe;
                while (lo < hi) {
                  const int mid = (lo + hi) >> 1;
                  if ((int64_t)a.set.sx[mid] < key) lo = mid + 1;
                  else hi = mid;
                }
                return lo;
              };
              int uH = qs, vH = qs, uL = qs, vL = qs;  // particle ranges: high part, low part
              if (X1 - X0 + 1 >= W) { uL = qs; vL = qe; }
              else if (X0 < 0) { uH = first_ge(X0 + W); vH = qe; uL = qs; vL = first_ge(X1 + 1); }
              else if (X1 >= W) { uH = first_ge(X0); vH = qe; uL = qs; vL = first_ge(X1 - W + 1); }
              else { uL = first_ge(X0); vL = first_ge(X1 + 1); }
              // to cluster ranges of the row (merged when both parts reach one cluster)
              int kL0 = 0, kL1 = -1, kH0 = 0, kH1 = -1;
              if (vL > uL) { kL0 = (uL - qs) / kClSize; kL1 = (vL - 1 - qs) / kClSize; }
              if (vH > uH) { kH0 = (uH - qs) / kClSize; kH1 = (vH - 1 - qs) / kClSize; }
              if (kL1 >= kL0 && kH1 >= kH0 && kL1 >= kH0 - 1) { kL1 = max(kL1, kH1); kH1 = kH0 - 1; }
              const int base = a.cl_base[r2i];
              if (kL1 >= kL0) {
                const int j0 = max(base + kL0, jmin), j1 = base + kL1;
                if (j1 >= j0) { b0 = j0; l0 = j1 - j0 + 1; }
              }
              if (kH1 >= kH0) {
                const int j0 = max(base + kH0, jmin), j1 = base + kH1;
                if (j1 >= j0) { b1 = j0; l1 = j1 - j0 + 1; }
              }
            }
          }
        }
        const int tot = l0 + l1;
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += v;
        }
        const int excl = carry + incl - tot;
        if (t < nrst) {
          seg_beg[2 * t] = b0;
          seg_pre[2 * t] = excl;
          seg_beg[2 * t + 1] = b1;
          seg_pre[2 * t + 1] = excl + l0;
        }
        carry += __shfl_sync(FULL, incl, 31);
      }
      if (lane == 0) seg_pre[2 * nrst] = carry;
      __syncwarp();
      const int T = carry;
      // Candidates in chunks of 32, one per lane: the box test against every i-cluster of
      // the group gives a mask; the warp then visits each candidate with a mask.
      int sg = 0;
      for (int base = 0; base < T; base += 32) {
        const int cc = base + lane;
        int s = sg, J = 0, jb = 0, jn = 0;
        uint32_t msk = 0u;
        float jy0 = 0.f, jz0 = 0.f;  // the candidate box's low corner in y and z (frame)
        if (cc < T) {
          while (seg_pre[s + 1] <= cc) ++s;
          J = seg_beg[s] + (cc - seg_pre[s]);
          const uint4 l = a.cl_lo[J], u = a.cl_hi[J];
          jb = (int)l.w;
          jn = (int)u.w;
          const float jx0 = (float)(int)(l.x - rx) * pc.h[0];
          jy0 = (float)(int)(l.y - ry) * pc.h[1];
          jz0 = (float)(int)(l.z - rz) * pc.h[2];
          const float jx1 = (float)(int)(u.x - rx) * pc.h[0];
          const float jy1 = (float)(int)(u.y - ry) * pc.h[1];
          const float jz1 = (float)(int)(u.z - rz) * pc.h[2];
          // a box that reaches past L/2 from the frame centre wraps (its ends swap sides): its
          // distance is then that of the nearer of its two pieces
          const bool wx = jx0 > jx1, wy = jy0 > jy1, wz = jz0 > jz1;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const float4 lo4 = ibl[c], hi4 = ibh[c];
            const float ax = jx0 - hi4.x, bx = lo4.x - jx1;
            const float ay = jy0 - hi4.y, by = lo4.y - jy1;
            const float az = jz0 - hi4.z, bz = lo4.z - jz1;
            const float gx = fmaxf(0.f, wx ? fminf(ax, bx) : fmaxf(ax, bx));
            const float gy = fmaxf(0.f, wy ? fminf(ay, by) : fmaxf(ay, by));
            const float gz = fmaxf(0.f, wz ? fminf(az, bz) : fmaxf(az, bz));
            const bool hit = c >= cb && c < ce && J >= g0 + c &&
                             fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= a.bb2;
            msk |= hit ? (1u << c) : 0u;
          }
        }
        sg = __shfl_sync(FULL, s, 31);
        unsigned vis = __ballot_sync(FULL, msk != 0u);
        while (vis) {
          const int t0 = __ffs(vis) - 1;
          vis &= vis - 1u;
          const int Jv = __shfl_sync(FULL, J, t0);
          const uint32_t M = __shfl_sync(FULL, msk, t0);
          const int vb = __shfl_sync(FULL, jb, t0), vn = __shfl_sync(FULL, jn, t0);
          const float cyj = F64 ? 0.f : __shfl_sync(FULL, jy0, t0);
          const float czj = F64 ? 0.f : __shfl_sync(FULL, jz0, t0);
          const int cdiag = Jv - g0;  // the visited cluster's place in the super-cluster
          // This lane's j particles, h and h + 4 of the cluster: x from the exact integer
          // offset from the frame centre, y and z from the cluster's corner plus the record's
          // offsets, in FP32 (exact integer offsets in the FP64 form).
          real xj[2], yj[2], zj[2], qj[2], fxj[2], fyj[2], fzj[2];
          int oxj[2], oyj[2], ozj[2], tj[2], cntj[2];
          bool vj[2];
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int t = hh + 4 * k;
            vj[k] = t < vn;
            const int p = vb + (vj[k] ? t : 0);
            oxj[k] = oyj[k] = ozj[k] = 0;
            qj[k] = (real)0;
            if (!F64) {
              // (an empty slot's y of -3e18 puts it out of reach)
              const uint4 pj = __ldg(&a.jrec[((int64_t)Jv << 3) + t]);
              xj[k] = (real)((float)(int)(pj.x - rx) * pc.h[0]);
              yj[k] = (real)(cyj + __uint_as_float(pj.y));
              zj[k] = (real)(czj + __uint_as_float(pj.z));
              if (COUL) qj[k] = (real)__uint_as_float(pj.w);
            } else {
              oxj[k] = (int)(a.set.sx[p] - rx);
              oyj[k] = (int)(a.set.sy[p] - ry);
              ozj[k] = (int)(a.set.sz[p] - rz);
              xj[k] = yj[k] = zj[k] = (real)0;
              if (COUL) qj[k] = (real)a.set.qd[p];
            }
            tj[k] = MULTI ? a.set.type[p] : 0;
            fxj[k] = fyj[k] = fzj[k] = (real)0;
            cntj[k] = 0;
          }
          float bmin = 3e38f;  // FP32 forms: smallest |r^2 - r_c^2| of the visit (band test)
          // Pair force of i (frame coordinates or integer offsets) with this lane's j particle k,
          // when `ok`; adds the reaction to j and returns the force factor and displacement.
          auto pair_one = [&](bool ok, real xi_, real yi_, real zi_, int oxi_, int oyi_,
                              int ozi_, real qi_, int ti_, int k, real &dx, real &dy, real &dz,
                              bool &in) -> real {
            real r2, ir2;
            if (F64) {
              // the offsets' difference (mod 2^32) is the exact minimum-image displacement
              const int dsx = (int)((uint32_t)oxi_ - (uint32_t)oxj[k]);
              const int dsy = (int)((uint32_t)oyi_ - (uint32_t)oyj[k]);
              const int dsz = (int)((uint32_t)ozi_ - (uint32_t)ozj[k]);
              dx = (real)__dmul_rn((double)dsx, pc.hd[0]);
              dy = (real)__dmul_rn((double)dsy, pc.hd[1]);
              dz = (real)__dmul_rn((double)dsz, pc.hd[2]);
              r2 = (real)__dadd_rn(__dadd_rn(__dmul_rn((double)dx, (double)dx),
                                             __dmul_rn((double)dy, (double)dy)),
                                   __dmul_rn((double)dz, (double)dz));
              in = ok && vj[k] && (double)r2 <= pc.rc2d;
              ir2 = in ? (real)(1.0 / (double)r2) : (real)0;
            } else {
              dx = xi_ - xj[k];
              dy = yi_ - yj[k];
              dz = zi_ - zj[k];
              r2 = (real)fmaf((float)dx, (float)dx, fmaf((float)dy, (float)dy, (float)(dz * dz)));
              in = ok && (float)r2 < pc.rc2_lo;
              bmin = fminf(bmin, fabsf((float)r2 - a.rc2_mid));
              ir2 = in ? (real)rcp_approx((float)r2) : (real)0;
            }
            const real g = cp_terms<real, COUL, MULTI>(a, in, r2, ir2, qi_, qj[k], ti_, tj[k], acc);
            fxj[k] = mad(-g, dx, fxj[k]); fyj[k] = mad(-g, dy, fyj[k]); fzj[k] = mad(-g, dz, fzj[k]);
            if (COUNT) cntj[k] += in ? 1 : 0;
            return g;
          };
          // The visited cluster may be one of the super-cluster's own (cdiag): its pairs with
          // itself count once (particle a8 with particle h + 4k > a8). They are taken here, with
          // the i particle read from shared memory and its force added by atomics, so that the
          // loop below carries no exclusion.
          uint32_t Mh = M;
          if (cdiag >= 0 && cdiag < NC && ((M >> cdiag) & 1u)) {
            Mh &= ~(1u << cdiag);
            const int t = kClSize * cdiag + a8;
            const bool vd = t < np && (asub < 0 || a8 == asub);
            const uint4 sd = si[t];
            const int ox = (int)(sd.x - rx), oy = (int)(sd.y - ry), oz = (int)(sd.z - rz);
            const real xd = vd ? (real)((float)ox * pc.h[0]) : (real)3e18f;
            const real yd = vd ? (real)((float)oy * pc.h[1]) : (real)3e18f;
            const real zd = vd ? (real)((float)oz * pc.h[2]) : (real)3e18f;
            real qd = (real)0;
            if (COUL) qd = F64 ? (vd ? (real)a.set.qd[p0 + t] : (real)0) : (real)__uint_as_float(sd.w);
            const int td = MULTI ? sti[t] : 0;
            real fdx = (real)0, fdy = (real)0, fdz = (real)0;
            int cd = 0;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              real dx, dy, dz;
              bool in;
              const real g = pair_one(vd && a8 < hh + 4 * k, xd, yd, zd, ox, oy, oz, qd, td, k,
                                      dx, dy, dz, in);
              fdx = mad(g, dx, fdx); fdy = mad(g, dy, fdy); fdz = mad(g, dz, fdz);
              if (COUNT) cd += in ? 1 : 0;
            }
            fdx += __shfl_xor_sync(FULL, fdx, 8); fdx += __shfl_xor_sync(FULL, fdx, 16);
            fdy += __shfl_xor_sync(FULL, fdy, 8); fdy += __shfl_xor_sync(FULL, fdy, 16);
            fdz += __shfl_xor_sync(FULL, fdz, 8); fdz += __shfl_xor_sync(FULL, fdz, 16);
            if (COUNT) {
              cd += __shfl_xor_sync(FULL, cd, 8);
              cd += __shfl_xor_sync(FULL, cd, 16);
            }
            if (vd && hh < 3) {
              const real v = hh == 0 ? fdx : (hh == 1 ? fdy : fdz);
              long long *dst = a.facc + (int64_t)hh * N + p0 + t;
              if (F64) fx_add(dst, (double)v, a.fscale_d, a.err);
              else fx_add(dst, (float)v, a.fscale, a.err);
            }
            if (COUNT && vd && hh == 3 && cd) atomicAdd(a.nbr + p0 + t, cd);
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if ((Mh >> c) & 1u) {
              const float4 pi4 = F64 ? make_float4(0.f, 0.f, 0.f, 0.f) : sif[kClSize * c + a8];
#pragma unroll
              for (int k = 0; k < 2; ++k) {
                real dx, dy, dz;
                bool in;
                const real g = pair_one(!F64 || vi[c], (real)pi4.x, (real)pi4.y, (real)pi4.z,
                                        oxi[c], oyi[c], ozi[c], COUL && !F64 ? (real)pi4.w : qi[c],
                                        ti[c], k, dx, dy, dz, in);
                fxi[c] = mad(g, dx, fxi[c]); fyi[c] = mad(g, dy, fyi[c]); fzi[c] = mad(g, dz, fzi[c]);
                if (COUNT) cnti[c] += in ? 1 : 0;
              }
            }
          }
          // Band pairs (FP32 forms): the exact decision; a pair inside is added by atomics.
          if (!F64 && __any_sync(FULL, bmin <= a.rc2_half)) {
            for (int c = cb; c < ce; ++c) {
              if (!((M >> c) & 1u)) continue;
              const int t = kClSize * c + a8;
              if (t >= np || (asub >= 0 && a8 != asub)) continue;
              const uint4 s = si[t];
              const float x0 = (float)(int)(s.x - rx) * pc.h[0];
              const float y0 = (float)(int)(s.y - ry) * pc.h[1];
              const float z0 = (float)(int)(s.z - rz) * pc.h[2];
              for (int k = 0; k < 2; ++k) {
                if (!vj[k] || !(c != cdiag || a8 < hh + 4 * k)) continue;
                const float dx = x0 - (float)xj[k], dy = y0 - (float)yj[k], dz = z0 - (float)zj[k];
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (!(r2 >= pc.rc2_lo && r2 <= pc.rc2_hi)) continue;
                const int pj = vb + hh + 4 * k;
                const int dsx = (int)(s.x - a.set.sx[pj]), dsy = (int)(s.y - a.set.sy[pj]),
                          dsz = (int)(s.z - a.set.sz[pj]);
                if (!(exact_r2(pc, dsx, dsy, dsz) <= pc.rc2d)) continue;
                const real qis = COUL ? (real)__uint_as_float(s.w) : (real)0;
                const real g = cp_terms<real, COUL, MULTI>(a, true, (real)r2, (real)rcp_approx(r2),
                                                           qis, qj[k], MULTI ? sti[t] : 0, tj[k],
                                                           acc);
                const int pi = p0 + t;
                fx_add(a.facc + pi, (float)(g * dx), a.fscale, a.err);
                fx_add(a.facc + N + pi, (float)(g * dy), a.fscale, a.err);
                fx_add(a.facc + 2 * N + pi, (float)(g * dz), a.fscale, a.err);
                fx_add(a.facc + pj, (float)(-g * dx), a.fscale, a.err);
                fx_add(a.facc + N + pj, (float)(-g * dy), a.fscale, a.err);
                fx_add(a.facc + 2 * N + pj, (float)(-g * dz), a.fscale, a.err);
                if (COUNT) { atomicAdd(a.nbr + pi, 1); atomicAdd(a.nbr + pj, 1); }
              }
            }
          }
          // Reaction on the visited cluster, reduce-scattered over the 8 lanes sharing h: of
          // the slots (fx, fy, fz of particle h, then of particle h + 4, then two zeros) lane
          // a8 ends with the sum of slot a8 over the 8 lanes and adds it (slots 0-5). The
          // exchange with lane a8 xor m (m = 1, 2, 4) pairs the slots that differ in bit m: a
          // lane keeps the one whose bit matches its own and adds its partner's copy of it,
          // so each sum is formed as the tree ((v_a + v_a^1) + (v_a^2 + v_a^3)) + (...) of a
          // full butterfly, with a third of its shuffles.
          {
            const bool b0 = a8 & 1, b1 = a8 & 2, b2 = a8 & 4;
            // xor 1: slot pairs (0, 1), (2, 3), (4, 5); w[p] holds slot 2p + b0 ((6, 7): zero)
            real w[3];
            {
              const real s0[3] = {fxj[0], fzj[0], fyj[1]}, s1[3] = {fyj[0], fxj[1], fzj[1]};
#pragma unroll
              for (int p = 0; p < 3; ++p)
                w[p] = (b0 ? s1[p] : s0[p]) + __shfl_xor_sync(FULL, b0 ? s0[p] : s1[p], 1);
            }
            // xor 2: (w0, w1) and (w2, 0); u[q] holds slot 4q + 2 b1 + b0
            const real u0 = (b1 ? w[1] : w[0]) + __shfl_xor_sync(FULL, b1 ? w[0] : w[1], 2);
            const real u1 = (b1 ? (real)0 : w[2]) + __shfl_xor_sync(FULL, b1 ? w[2] : (real)0, 2);
            // xor 4: slot a8
            const real v = (b2 ? u1 : u0) + __shfl_xor_sync(FULL, b2 ? u0 : u1, 4);
            if (a8 < 6) {
              const int k = a8 / 3, d = a8 - 3 * k;
              if (vj[k]) {
                long long *dst = a.facc + (int64_t)d * N + vb + hh + 4 * k;
                if (F64) fx_add(dst, (double)v, a.fscale_d, a.err);
                else fx_add(dst, (float)v, a.fscale, a.err);
              }
            }
          }
          if (COUNT) {
            const unsigned gm = 0xffu << (8 * hh);
            const int c0 = __reduce_add_sync(gm, cntj[0]);
            const int c1 = __reduce_add_sync(gm, cntj[1]);
            if (a8 == 0) {
              if (vj[0] && c0) atomicAdd(a.nbr + vb + hh, c0);
              if (vj[1] && c1) atomicAdd(a.nbr + vb + hh + 4, c1);
            }
          }
        }
      }
      // i forces: sum over the four lanes sharing a8, then lane (h, a8) adds clusters c with
      // c % 4 == h
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        fxi[c] += __shfl_xor_sync(FULL, fxi[c], 8); fxi[c] += __shfl_xor_sync(FULL, fxi[c], 16);
        fyi[c] += __shfl_xor_sync(FULL, fyi[c], 8); fyi[c] += __shfl_xor_sync(FULL, fyi[c], 16);
        fzi[c] += __shfl_xor_sync(FULL, fzi[c], 8); fzi[c] += __shfl_xor_sync(FULL, fzi[c], 16);
        if (COUNT) {
          cnti[c] += __shfl_xor_sync(FULL, cnti[c], 8);
          cnti[c] += __shfl_xor_sync(FULL, cnti[c], 16);
        }
        const int t = kClSize * c + a8;
        if ((c & 3) == hh && vi[c]) {
          const int64_t pi = p0 + t;
          if (F64) {
            fx_add(a.facc + pi, (double)fxi[c], a.fscale_d, a.err);
            fx_add(a.facc + N + pi, (double)fyi[c], a.fscale_d, a.err);
            fx_add(a.facc + 2 * N + pi, (double)fzi[c], a.fscale_d, a.err);
          } else {
            fx_add(a.facc + pi, (float)fxi[c], a.fscale, a.err);
            fx_add(a.facc + N + pi, (float)fyi[c], a.fscale, a.err);
            fx_add(a.facc + 2 * N + pi, (float)fzi[c], a.fscale, a.err);
          }
          if (COUNT && cnti[c]) atomicAdd(a.nbr + pi, cnti[c]);
        }
      }
      __syncwarp();
      if (asub < 0) {
        cb = ce;
      } else if (++asub >= min(kClSize, np - kClSize * cb)) {
        asub = -1;
        ++cb;
      }
    }
  }
  // block partials of the energies and virials (each pair counted once)
  double ulj, wlj;
  if (MULTI) {
    ulj = (double)acc.u0;
    wlj = (double)acc.u1;
  } else {
    const double A = F64 ? a.ljAd : (double)a.ljA, B = F64 ? a.ljBd : (double)a.ljB;
    ulj = A * (double)acc.u0 - B * (double)acc.u1;
    wlj = 12.0 * A * (double)acc.u0 - 6.0 * B * (double)acc.u1;
  }
  double v[NQ_PAIR] = {(double)acc.uc - (double)acc.cuc, ulj, (double)acc.wc - (double)acc.cwc, wlj};
#pragma unroll
  for (int k = 0; k < NQ_PAIR; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) a.epart[(int64_t)bx * NQ_PAIR + k] = s;
  }
  // the pass's partial slots past the grid (the range is sized for the per-particle kernel,
  // the grid for the super-clusters) hold zeros
  for (int64_t z = (int64_t)bx + nbx; z < a.nslots; z += nbx)
    if (lane < NQ_PAIR) a.epart[z * NQ_PAIR + lane] = 0.0;
}

// (occupancy: 24 warps per SM for the FP32 LJ pass, fewer for the register-heavy Coulomb and
// FP64 instances)
#ifndef RBE_CP_MINB
#define RBE_CP_MINB 24
#endif
#define RBE_CP_BOUNDS                                                                          \
  __launch_bounds__(32, (sizeof(real) == 8 ? (COUL ? 8 : 12) : (COUL ? 12 : RBE_CP_MINB)))
template <typename real, bool COUL, bool MULTI, bool COUNT>
__global__ void RBE_CP_BOUNDS cpair_kernel(const ClusterArgs a) {
  cpair_body<real, COUL, MULTI, COUNT>(a, (int)blockIdx.x, (int)gridDim.x);
}
#undef RBE_CP_BOUNDS

// ---------------------------------------------------------------------------------------
// Host side

int cpair_nc(const Ctx &c) { return c.precision == RBE_FP64 ? 4 : 8; }

// Upper bound of the super-clusters of N particles in the rows of the grid.
int64_t cpair_blocks_bound(const Ctx &c) {
  const int64_t nrows = (int64_t)c.grid.n[1] * c.grid.n[2];
  return c.N / (kClSize * cpair_nc(c)) + nrows + 1;
}
int64_t cpair_clusters_bound(const Ctx &c) {
  const int64_t nrows = (int64_t)c.grid.n[1] * c.grid.n[2];
  return c.N / kClSize + nrows + 1;
}

// The cluster kernel applies when a super-cluster's frame is a valid minimum image for y
// and z (one cell width plus 2 r_c below L) and a group of at least one typical cluster
// fits in x, with a stencil of at most 3 cells.
bool cpair_usable(const Ctx &c) {
  if (c.rbl || !c.pair_cluster) return false;
  for (int d = 1; d < 3; ++d) {
    if (c.grid.R[d] > 3) return false;
    const double w = c.box[d] / c.grid.n[d];
    if (!(w + 2.0 * c.rc < c.box[d] * (1.0 - 1e-9))) return false;
  }
  // room in x for at least a few cells' worth of a group
  return c.box[0] - 2.0 * c.rc > 2.0 * c.box[0] / c.grid.n[0];
}

cudaError_t launch_cluster_tables(Ctx &c) {
  const int b = c.cur;
  const int nrows = c.grid.n[1] * c.grid.n[2];
  const RowsArgs ra{c.cell_start, c.grid.n[0], nrows, cpair_nc(c), c.cl_base, c.sc_base};
  cudaError_t e = dispatch(c, cluster_rows_kernel, cluster_rows_kernel_b, dim3(1), dim3(1024), 0,
                           ra);
  if (e != cudaSuccess) return e;
  const int64_t ccap = cpair_clusters_bound(c);
  const BoundsArgs ba{c.s[b], c.s[b] + c.N, c.s[b] + 2 * c.N, c.qf[b], c.cell_start, c.grid.n[0],
                      nrows, c.cl_base, ccap, c.cl_lo, c.cl_hi, c.cjrec, c.pc.h[1], c.pc.h[2]};
  return dispatch(c, cluster_bounds_kernel, cluster_bounds_kernel_b,
                  dim3((unsigned)((kClSize * ccap + 255) / 256)), dim3(256), 0, ba);
}

// The pair pass itself (the tables of launch_cluster_tables must be current); its forces stay
// in the fixed-point sums, which the Coulomb pass and the k-space gather add to before
// launch_cluster_finish converts them.
cudaError_t launch_cluster_pair(Ctx &c, bool coul, bool multi, bool want_counts) {
  const int b = c.cur;
  const int nrows = c.grid.n[1] * c.grid.n[2];
  ClusterArgs a;
  a.set.sx = c.s[b]; a.set.sy = c.s[b] + c.N; a.set.sz = c.s[b] + 2 * c.N;
  a.set.qf = c.qf[b]; a.set.qd = c.qd[b]; a.set.type = c.type[b];
  a.set.cell_start = c.cell_start; a.set.map = nullptr; a.set.n = c.N;
  a.grid = c.grid;
  a.pc = c.pc;
  a.ljA = c.lj.A[0]; a.ljB = c.lj.B[0]; a.ljA12 = c.lj.A12[0]; a.ljB6 = c.lj.B6[0];
  a.ljAd = c.lj.Ad[0]; a.ljBd = c.lj.Bd[0]; a.ljA12d = c.lj.A12d[0]; a.ljB6d = c.lj.B6d[0];
  a.table = reinterpret_cast<const LJTable *>(c.lj_dev);
  a.cl_base = c.cl_base; a.sc_base = c.sc_base; a.cl_lo = c.cl_lo; a.cl_hi = c.cl_hi;
  a.jrec = c.cjrec;
  a.nrows = nrows;
  a.facc = c.facc;
  a.N = c.N;
  a.fscale = (float)kFixScale32;
  a.fscale_d = kFixScale64;
  a.epart = c.epart + c.off_pair;
  a.nbr = want_counts ? c.nbr : nullptr;
  a.comp = c.precision == RBE_FP32_COMP;
  {
    // x extent of a group: (extent + 2 r_c) < L, in fractional units, with margin
    const double lim = (c.box[0] - 2.0 * c.rc) / c.box[0] * kTwo32 * (1.0 - 1e-7) - 16.0;
    a.xlim = (uint32_t)std::max(0.0, std::min(lim, 4294967295.0));
    // frame coordinates within L/2 on every axis: the exact-decision band for that extent.
    // A j particle's y and z add one more rounding (corner plus offset: within 3u |y| + 4u w
    // for a cell width w, against the 2u |y| the band assumes per coordinate); extents
    // raised by 2 r_c + 2 w cover it, as |y| <= L/2.
    double X[3];
    for (int d = 0; d < 3; ++d) X[d] = 0.5 * c.box[d];
    for (int d = 1; d < 3; ++d) X[d] += 2.0 * c.rc + 2.0 * c.box[d] / c.grid.n[d];
    const double band = frame_band(X, c.rc, c.box, false);
    a.pc.rc2_lo = (float)(c.rc * c.rc * (1.0 - band));
    a.pc.rc2_hi = (float)(c.rc * c.rc * (1.0 + band));
    // band test |r^2 - mid| <= half: half reaches past both FP32 edges by a few ulps (the
    // edges are rounded to FP32; the difference r^2 - mid is exact near mid)
    a.rc2_mid = (float)(c.rc * c.rc);
    const double mid = a.rc2_mid, ulp = std::nextafter((float)mid, 3e38f) - (float)mid;
    a.rc2_half = (float)(std::max((double)a.pc.rc2_hi - mid, mid - (double)a.pc.rc2_lo) + 4.0 * ulp);
    // box test: squared gap of FP32 frame boxes (each bound within 2u L/2, the gap within
    // u L more), widened so that no pair within r_c is lost
    const double u = std::ldexp(1.0, -24);
    double e = 0.0;
    for (int d = 0; d < 3; ++d) e = std::max(e, 3.0 * u * c.box[d]);
    const double rr = c.rc * (1.0 + 1e-5) + 2.0 * e;
    a.bb2 = (float)(rr * rr);
  }
  a.err = c.err;
  if (want_counts) {
    const cudaError_t e = fill_zero(c, c.nbr, c.N);
    if (e != cudaSuccess) return e;
  }
  // a block per possible super-cluster (blocks past the last one, and each block for the
  // slots past the grid, write zeros to the pass's partial range)
  a.nslots = c.n_pair_blk;
  const dim3 g((unsigned)std::min<int64_t>(c.n_pair_blk, cpair_blocks_bound(c))), bl(32);
  const bool fp64 = c.precision == RBE_FP64;
  cudaError_t e;
  // (per replica in a batch)
#define RBE_CP_LAUNCH(R, CO, MU)                                                             \
  e = want_counts ? dispatch(c, cpair_kernel<R, CO, MU, true>, nullptr, g, bl, 0, a, true)   \
                  : dispatch(c, cpair_kernel<R, CO, MU, false>, nullptr, g, bl, 0, a, true)
  if (fp64) {
    if (coul) { if (multi) RBE_CP_LAUNCH(double, true, true); else RBE_CP_LAUNCH(double, true, false); }
    else { if (multi) RBE_CP_LAUNCH(double, false, true); else RBE_CP_LAUNCH(double, false, false); }
  } else {
    if (coul) { if (multi) RBE_CP_LAUNCH(float, true, true); else RBE_CP_LAUNCH(float, true, false); }
    else { if (multi) RBE_CP_LAUNCH(float, false, true); else RBE_CP_LAUNCH(float, false, false); }
  }
#undef RBE_CP_LAUNCH
  return e;
}

// F = the fixed-point sums / scale, and the sums cleared for the next step.
cudaError_t launch_cluster_finish(Ctx &c) {
  const bool fp64 = c.precision == RBE_FP64;
  const int64_t n3 = 3 * c.N;
  // (per replica in a batch too: it joins the pair kernel, the Coulomb pass and the gather in
  // one run of per-replica launches, one fork and join per step)
  const dim3 fg((unsigned)(((n3 + 3) / 4 + 255) / 256)), fb(256);
  if (fp64) {
    const FinishArgs f{c.facc, c.Fd, n3, 0.f, 0.f, 1.0 / kFixScale64};
    return dispatch(c, cpair_finalize_kernel<double>, cpair_finalize_kernel_b<double>, fg, fb, 0, f,
                    true);
  }
  const FinishArgs f{c.facc, c.F, n3, (float)(4294967296.0 / kFixScale32),
                     (float)(1.0 / kFixScale32), 0.0};
  return dispatch(c, cpair_finalize_kernel<float>, cpair_finalize_kernel_b<float>, fg, fb, 0, f,
                  true);
}

}  // namespace rbe
