// k_list.cu -- Verlet neighbour list with skin for the real-space pair forces (Eqs. F_i,
// G_short, LJ), the short-range traversal of Sec. 3.1 that RBE is combined with.
//
// A list built at r_list = r_c + skin holds, for every i, each j with r_ij <= r_list at the
// time of the build. It stays complete for r_c while no particle has moved by skin / 2 or
// more since then: a pair with r_ij <= r_c now was closer than r_c + skin at the build.
// Each force evaluation first measures every displacement from the build positions
// (exactly, from the fixed-point coordinates; the FP32 test is conservative) and raises a
// device flag when one reaches skin / 2 (x (1 - 1e-5)); the cell sort and the list build
// run only on that flag, inside the same graph, so no host round trip decides a rebuild.
// Between builds the particle order is fixed (the list stores sorted slots).
//
// The evaluation kernel takes one thread per particle i and walks its list, warp-
// interleaved (entry t of slot i at list[((i / 32) * K + t) * 32 + i % 32], one coalesced
// 128-byte line per warp and entry). Candidates are gathered as packed (s_x, s_y, s_z, q)
// and go through the same exact cutoff decision as the cell kernel, so neighbour counts
// are bit-exact against the oracle; pairs between r_c and r_list contribute nothing.
#include <algorithm>

#include "pair_common.cuh"

namespace rbe {

// Device list flags (int32): [0] rebuild this step, [1] rebuild forced (new positions or
// list just enabled), [2] / [3] longest list of the running build (full / charged set),
// [4] / [5] longest list of the last finished build.
__global__ void __launch_bounds__(256)
    vl_check_kernel(const uint32_t *__restrict__ s, const uint32_t *__restrict__ ref,
                    int64_t N, float hx, float hy, float hz, float lim2,
                    int32_t *__restrict__ flags, unsigned long long *__restrict__ counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool moved = false;
  if (i < N) {
    const float dx = (float)(int)(s[i] - ref[i]) * hx;
    const float dy = (float)(int)(s[N + i] - ref[N + i]) * hy;
    const float dz = (float)(int)(s[2 * N + i] - ref[2 * N + i]) * hz;
    moved = mad(dx, dx, mad(dy, dy, dz * dz)) >= lim2;
  }
  if (__any_sync(0xffffffffu, moved) && (threadIdx.x & 31) == 0) atomicOr(&flags[0], 1);
  if (i == 0) {
    if (flags[1]) atomicOr(&flags[0], 1);
    counts[1] += 1;  // force evaluations since the list was enabled
  }
}

// After a build: the build positions become the reference, the forced flag clears, the
// longest lists are published and their running maxima reset.
__global__ void __launch_bounds__(256)
    vl_commit_kernel(const uint32_t *__restrict__ s, uint32_t *__restrict__ ref, int64_t n3,
                     int32_t *__restrict__ flags, unsigned long long *__restrict__ counts) {
  if (flags[0] == 0) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n3) ref[k] = s[k];
  if (k == 0) {
    flags[1] = 0;
    flags[4] = flags[2];
    flags[5] = flags[3];
    flags[2] = 0;
    flags[3] = 0;
    counts[0] += 1;  // builds
  }
}

struct ListArgs {
  PairArgs pa;        // set, constants, outputs; pa.list / pa.len / pa.K: the list
  const uint4 *s4;    // packed (s_x, s_y, s_z, q bits) of the set, sorted order
};

constexpr int kListUnroll = 4;

template <typename real, bool LJ, bool COUL, bool MULTI>
__global__ void __launch_bounds__(kPairWarps * 32) list_pair_kernel(const ListArgs la) {
  __shared__ double wred[kPairWarps][NQ_PAIR];
  const PairArgs &a = la.pa;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const int64_t n = a.set.n;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  const LJTable *tab = a.table;
  PairAcc<real> acc;
  acc.fx = acc.fy = acc.fz = acc.ulj = acc.wlj = acc.uc = acc.wc = (real)0;
  acc.cuc = acc.cwc = (real)0;
  acc.nbr = 0;
  const uint4 pi = valid ? la.s4[i] : make_uint4(0u, 0u, 0u, 0u);
  real qi = (real)0;
  if (COUL && valid) qi = sizeof(real) == 8 ? (real)a.set.qd[i] : (real)__uint_as_float(pi.w);
  const int ti = (MULTI && valid) ? a.set.type[i] : 0;
  const int len = valid ? a.len[i] : 0;
  const int lmax = __reduce_max_sync(FULL, len);
  const int32_t *L = a.list + (i >> 5) * (int64_t)a.K * 32 + lane;
  for (int t = 0; t < lmax; t += kListUnroll) {
    int jj[kListUnroll];
    bool ac[kListUnroll];
#pragma unroll
    for (int u = 0; u < kListUnroll; ++u) {
      ac[u] = t + u < len;
      jj[u] = ac[u] ? __ldcs(L + (int64_t)(t + u) * 32) : 0;  // the list streams once
    }
    uint4 pj[kListUnroll];
#pragma unroll
    for (int u = 0; u < kListUnroll; ++u) pj[u] = __ldg(&la.s4[jj[u]]);
#pragma unroll
    for (int u = 0; u < kListUnroll; ++u) {
      real qj = (real)0;
      if (COUL) qj = sizeof(real) == 8 ? (real)a.set.qd[jj[u]] : (real)__uint_as_float(pj[u].w);
      const int tj = MULTI ? a.set.type[jj[u]] : 0;
      pair_eval_masked<real, LJ, COUL, MULTI>(a, tab, ac[u], (int)(pi.x - pj[u].x),
                                              (int)(pi.y - pj[u].y), (int)(pi.z - pj[u].z),
                                              qi, ti, qj, tj, acc);
    }
  }
  if (valid) {
    const int64_t o = a.set.map ? (int64_t)a.set.map[i] : i;
    const int64_t S = a.Fstride;
    if (sizeof(real) == 8) {
      if (a.accumulate) { a.Fd[o] += (double)acc.fx; a.Fd[S + o] += (double)acc.fy; a.Fd[2 * S + o] += (double)acc.fz; }
      else { a.Fd[o] = (double)acc.fx; a.Fd[S + o] = (double)acc.fy; a.Fd[2 * S + o] = (double)acc.fz; }
    } else {
      if (a.accumulate) { a.F[o] += (float)acc.fx; a.F[S + o] += (float)acc.fy; a.F[2 * S + o] += (float)acc.fz; }
      else { a.F[o] = (float)acc.fx; a.F[S + o] = (float)acc.fy; a.F[2 * S + o] = (float)acc.fz; }
    }
    if (a.nbr) a.nbr[i] = acc.nbr;
  }
  double v[NQ_PAIR] = {(double)acc.uc - (double)acc.cuc, (double)acc.ulj,
                       (double)acc.wc - (double)acc.cwc, (double)acc.wlj};
#pragma unroll
  for (int k = 0; k < NQ_PAIR; ++k) {
    const double w = warp_sum(v[k]);
    if (lane == 0) wred[wid][k] = w;
  }
  __syncthreads();
  if (threadIdx.x < NQ_PAIR) {
    double s = 0.0;
    for (int w = 0; w < kPairWarps; ++w) s += wred[w][threadIdx.x];
    a.epart[(int64_t)blockIdx.x * NQ_PAIR + threadIdx.x] = 0.5 * s;
  }
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_list_check(Ctx &c) {
  const int b = c.cur;
  cudaError_t e = cudaMemsetAsync(c.vl_flags, 0, sizeof(int32_t), c.stream);
  if (e != cudaSuccess) return e;
  const double half = 0.5 * c.vl_skin;
  const float lim2 = (float)(half * half * (1.0 - 1e-5));
  vl_check_kernel<<<nblk(std::max<int64_t>(c.N, 1), 256), 256, 0, c.stream>>>(
      c.s[b], c.vl_ref, c.N, c.pc.h[0], c.pc.h[1], c.pc.h[2], lim2, c.vl_flags, c.vl_count);
  return cudaGetLastError();
}

cudaError_t launch_list_commit(Ctx &c) {
  const int64_t n3 = 3 * c.N;
  vl_commit_kernel<<<nblk(std::max<int64_t>(n3, 1), 256), 256, 0, c.stream>>>(
      c.s[c.cur], c.vl_ref, n3, c.vl_flags, c.vl_count);
  return cudaGetLastError();
}

template <typename real, bool LJ, bool COUL>
static void list_launch(const ListArgs &la, int64_t n, bool multi, cudaStream_t st) {
  if (n == 0) return;
  const dim3 g(nblk(n, kPairWarps * 32)), b(kPairWarps * 32);
  if (multi) list_pair_kernel<real, LJ, COUL, true><<<g, b, 0, st>>>(la);
  else list_pair_kernel<real, LJ, COUL, false><<<g, b, 0, st>>>(la);
}

// Pair forces from the lists: one pass over all particles (LJ, and Coulomb when most
// particles are charged), then the Coulomb pass over the charged subset's own lists.
cudaError_t launch_list_pair(Ctx &c, bool want_counts) {
  const int b = c.cur;
  const bool fused = c.Nq * 2 > c.N;
  const bool multi = c.nt > 1;
  const bool fp64 = c.precision == RBE_FP64;
  ListArgs la{};
  PairArgs &a = la.pa;
  a.grid = c.grid;
  a.pc = c.pc;
  a.ljA = c.lj.A[0]; a.ljB = c.lj.B[0]; a.ljA12 = c.lj.A12[0]; a.ljB6 = c.lj.B6[0];
  a.ljAd = c.lj.Ad[0]; a.ljBd = c.lj.Bd[0]; a.ljA12d = c.lj.A12d[0]; a.ljB6d = c.lj.B6d[0];
  a.table = reinterpret_cast<const LJTable *>(c.lj_dev);
  a.F = c.F; a.Fd = c.Fd; a.Fstride = c.N;
  a.set.sx = c.s[b]; a.set.sy = c.s[b] + c.N; a.set.sz = c.s[b] + 2 * c.N;
  a.set.qf = c.qf[b]; a.set.qd = c.qd[b]; a.set.type = c.type[b];
  a.set.cell_start = nullptr; a.set.map = nullptr; a.set.n = c.N;
  a.accumulate = 0;
  a.epart = c.epart + c.off_pair;
  a.nbr = want_counts ? c.nbr : nullptr;
  a.comp = c.precision == RBE_FP32_COMP;
  a.list = c.vl_list; a.len = c.vl_len; a.K = c.vl_K;
  la.s4 = c.s4;
  if (fused) {
    if (fp64) list_launch<double, true, true>(la, c.N, multi, c.stream);
    else list_launch<float, true, true>(la, c.N, multi, c.stream);
  } else {
    if (fp64) list_launch<double, true, false>(la, c.N, multi, c.stream);
    else list_launch<float, true, false>(la, c.N, multi, c.stream);
  }
  zero_partials_tail(c, c.off_pair, nblk(c.N, kPairWarps * 32), c.n_pair_blk);
  mark(c, RBE_PH_PAIR2);
  if (!fused && c.Nq > 0) {
    ListArgs lq = la;
    PairArgs &q = lq.pa;
    q.set.sx = c.cs; q.set.sy = c.cs + c.Nq; q.set.sz = c.cs + 2 * c.Nq;
    q.set.qf = c.cqf; q.set.qd = c.cqd; q.set.type = nullptr;
    q.set.map = c.cmap; q.set.n = c.Nq;
    q.accumulate = 1;
    q.epart = c.epart + c.off_coul;
    q.nbr = nullptr;
    q.list = c.vl_listq; q.len = c.vl_lenq; q.K = c.vl_Kq;
    lq.s4 = c.cs4;
    if (fp64) list_launch<double, false, true>(lq, c.Nq, false, c.stream);
    else list_launch<float, false, true>(lq, c.Nq, false, c.stream);
    zero_partials_tail(c, c.off_coul, nblk(c.Nq, kPairWarps * 32), c.n_coul_blk);
  }
  return cudaGetLastError();
}

}  // namespace rbe
