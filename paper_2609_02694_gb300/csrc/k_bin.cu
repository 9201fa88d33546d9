// k_bin.cu -- linked-cell binning and cell-wise reordering (Sec. 2.2: "linked-cell
// reassignment and cell-wise reordering").
//
// Cell of a particle: c_d = floor(s_d n_d / 2^32) (exact on the fixed-point grid),
// c = c_x + n_x (c_y + n_y c_z). Particles are reordered by (cell, s_x, id), which is
// unique, so the order (and every sum taken in it) is independent of the previous order and
// of atomic timing, and every row of cells is sorted by x. The charged subset is reordered
// the same way into its own arrays.
// Pipeline: count (atomics give a provisional slot) -> exclusive scan of the counts ->
// provisional scatter -> per-cell rank by key + permute of every field (warps per cells).
// Integer work, HBM-bound.
// With a Verlet neighbour list the order must stay fixed between list builds: every kernel
// of the pipeline then reads a device gate (1 = rebuild this step) and returns at once when
// it is 0, and an identity copy into the other buffer runs instead, so the buffers still
// alternate every step. Both paths also write the packed (s_x, s_y, s_z, q) copies the list
// kernels gather from.
#include <climits>

#include "rbe_internal.cuh"

namespace rbe {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanBlock = kScanThreads * kScanItems;

// true when a gated kernel has nothing to do this step
__device__ __forceinline__ bool gated_off(const int32_t *gate) { return gate && *gate == 0; }

struct CountArgs {
  int64_t N;
  const uint32_t *s;
  const float *q;
  int n0, n1, n2;
  int32_t *count, *ccount, *key, *off;
  const int32_t *gate;
};

__device__ __forceinline__ void bin_count_body(const CountArgs &a, int bx, int) {
  const int64_t i = (int64_t)bx * blockDim.x + threadIdx.x;
  const int64_t N = a.N;
  if (i >= N || gated_off(a.gate)) return;
  const int cx = cell_of(a.s[i], a.n0), cy = cell_of(a.s[N + i], a.n1),
            cz = cell_of(a.s[2 * N + i], a.n2);
  const int c = cx + a.n0 * (cy + a.n1 * cz);
  a.key[i] = c;
  a.off[i] = atomicAdd(&a.count[c], 1);
  if (a.q[i] != 0.0f) atomicAdd(&a.ccount[c], 1);
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), bin_count_kernel, CountArgs, bin_count_body)

// N a multiple of 4: four consecutive particles a thread in 16-byte accesses (the arrays
// start 256-byte aligned). The provisional slots the atomics hand out do not reach the final
// order, which the permute takes from the (cell, s_x, id) keys.
__device__ __forceinline__ void bin_count4_body(const CountArgs &a, int bx, int) {
  const int64_t i = 4 * ((int64_t)bx * blockDim.x + threadIdx.x);
  const int64_t N = a.N;
  if (i >= N || gated_off(a.gate)) return;
  const uint4 sx = *reinterpret_cast<const uint4 *>(a.s + i);
  const uint4 sy = *reinterpret_cast<const uint4 *>(a.s + N + i);
  const uint4 sz = *reinterpret_cast<const uint4 *>(a.s + 2 * N + i);
  const float4 q = *reinterpret_cast<const float4 *>(a.q + i);
  auto key = [&](uint32_t x, uint32_t y, uint32_t z) {
    return cell_of(x, a.n0) + a.n0 * (cell_of(y, a.n1) + a.n1 * cell_of(z, a.n2));
  };
  const int4 c = make_int4(key(sx.x, sy.x, sz.x), key(sx.y, sy.y, sz.y), key(sx.z, sy.z, sz.z),
                           key(sx.w, sy.w, sz.w));
  *reinterpret_cast<int4 *>(a.key + i) = c;
  int4 o;
  o.x = atomicAdd(&a.count[c.x], 1);
  o.y = atomicAdd(&a.count[c.y], 1);
  o.z = atomicAdd(&a.count[c.z], 1);
  o.w = atomicAdd(&a.count[c.w], 1);
  *reinterpret_cast<int4 *>(a.off + i) = o;
  if (q.x != 0.0f) atomicAdd(&a.ccount[c.x], 1);
  if (q.y != 0.0f) atomicAdd(&a.ccount[c.y], 1);
  if (q.z != 0.0f) atomicAdd(&a.ccount[c.z], 1);
  if (q.w != 0.0f) atomicAdd(&a.ccount[c.w], 1);
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), bin_count4_kernel, CountArgs, bin_count4_body)

// Arguments of the three scan passes and the provisional scatter.
struct ScanArgs {
  const int32_t *cnt;
  int32_t *start, *blk;
  int64_t ncell, nblk;
  const int32_t *gate;
};
struct ScatterArgs {
  int64_t N;
  const int32_t *key, *off, *start;
  int32_t *tmp;
  const int32_t *gate;
};

// Exclusive scan, three passes. Arrays hold two independent sequences (blockIdx.y).
__device__ __forceinline__ void scan_block_body(const ScanArgs &a, int bx, int) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  if (gated_off(a.gate)) return;
  const int64_t ncell = a.ncell, nblk = a.nblk;
  const int which = blockIdx.y;
  const int32_t *in = a.cnt + which * ncell;
  int32_t *out = a.start + which * (ncell + 1);
  const int64_t base = (int64_t)bx * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t tsum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t idx = base + k;
    v[k] = idx < ncell ? in[idx] : 0;
    tsum += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive
  }
  __syncthreads();
  int32_t run = warp_tot[wid] + incl - tsum;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t idx = base + k;
    if (idx < ncell) out[idx] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) a.blk[which * nblk + bx] = run;  // block total
}
RBE_BATCHED_KERNEL(__launch_bounds__(kScanThreads), scan_block_kernel, ScanArgs, scan_block_body)

// One block per sequence.
__device__ __forceinline__ void scan_top_body(const ScanArgs &a, int bx, int) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry_s;
  if (gated_off(a.gate)) return;
  const int64_t ncell = a.ncell, nblk = a.nblk;
  const int which = bx;
  int32_t *b = a.blk + which * nblk;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base < nblk; base += 1024) {
    const int64_t idx = base + threadIdx.x;
    const int32_t v = idx < nblk ? b[idx] : 0;
    int32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const int32_t w = warp_tot[lane];
      int32_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      warp_tot[lane] = wi - w;
    }
    __syncthreads();
    const int32_t carry = carry_s;
    const int32_t excl = carry + warp_tot[wid] + incl - v;
    if (idx < nblk) b[idx] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) a.start[which * (ncell + 1) + ncell] = carry_s;
}
RBE_BATCHED_KERNEL(__launch_bounds__(1024), scan_top_kernel, ScanArgs, scan_top_body)

__device__ __forceinline__ void scan_add_body(const ScanArgs &a, int bx, int) {
  if (gated_off(a.gate)) return;
  const int64_t ncell = a.ncell;
  const int which = blockIdx.y;
  int32_t *out = a.start + which * (ncell + 1);
  const int32_t add = a.blk[which * a.nblk + bx];
  const int64_t base = (int64_t)bx * kScanBlock;
  for (int k = threadIdx.x; k < kScanBlock; k += kScanThreads) {
    const int64_t idx = base + k;
    if (idx < ncell) out[idx] += add;
  }
}
RBE_BATCHED_KERNEL(__launch_bounds__(kScanThreads), scan_add_kernel, ScanArgs, scan_add_body)

__device__ __forceinline__ void bin_scatter_body(const ScatterArgs &a, int bx, int) {
  const int64_t i = (int64_t)bx * blockDim.x + threadIdx.x;
  if (i >= a.N || gated_off(a.gate)) return;
  a.tmp[a.start[a.key[i]] + a.off[i]] = (int32_t)i;
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), bin_scatter_kernel, ScatterArgs, bin_scatter_body)

// N a multiple of 4: four consecutive particles a thread
__device__ __forceinline__ void bin_scatter4_body(const ScatterArgs &a, int bx, int) {
  const int64_t i = 4 * ((int64_t)bx * blockDim.x + threadIdx.x);
  if (i >= a.N || gated_off(a.gate)) return;
  const int4 k = *reinterpret_cast<const int4 *>(a.key + i);
  const int4 o = *reinterpret_cast<const int4 *>(a.off + i);
  const int32_t s0 = a.start[k.x], s1 = a.start[k.y], s2 = a.start[k.z], s3 = a.start[k.w];
  a.tmp[s0 + o.x] = (int32_t)i;
  a.tmp[s1 + o.y] = (int32_t)(i + 1);
  a.tmp[s2 + o.z] = (int32_t)(i + 2);
  a.tmp[s3 + o.w] = (int32_t)(i + 3);
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), bin_scatter4_kernel, ScatterArgs, bin_scatter4_body)

struct PermuteArgs {
  int64_t N, Nq, ncell;
  const int32_t *cell_start, *ccell_start, *tmp;
  const uint32_t *s0; uint32_t *s1;
  const float *vf0; float *vf1;
  const double *vd0; double *vd1;
  const int32_t *id0; int32_t *id1;
  const float *qf0; float *qf1;
  const double *qd0; double *qd1;
  const int32_t *ty0; int32_t *ty1;
  const float *im0; float *im1;
  uint32_t *cs; float *cqf; double *cqd; int32_t *cmap;
  uint4 *s4, *cs4;        // packed (s_x, s_y, s_z, q bits) copies, nullable
  const int32_t *gate;    // nullable: always run
};

// Within-cell order key (s_x, id): every row of cells is then sorted by x, and the pair and
// RBL kernels trim each row's run to the x-range their group can reach.
__device__ __forceinline__ uint64_t member_key(const PermuteArgs &a, int32_t o, int32_t id) {
  return ((uint64_t)a.s0[o] << 32) | (uint32_t)id;
}

// Move every field of the particle in provisional slot o to its final slot p (and, when
// charged, to charged slot pc of the charged subset).
__device__ __forceinline__ void move_particle(const PermuteArgs &a, int32_t o, int64_t p,
                                              int32_t myid, bool mych, int64_t pc) {
  const int64_t N = a.N, Nq = a.Nq;
  const uint32_t sx = a.s0[o], sy = a.s0[N + o], sz = a.s0[2 * N + o];
  a.s1[p] = sx; a.s1[N + p] = sy; a.s1[2 * N + p] = sz;
  if (a.vf0) { a.vf1[p] = a.vf0[o]; a.vf1[N + p] = a.vf0[N + o]; a.vf1[2 * N + p] = a.vf0[2 * N + o]; }
  if (a.vd0) { a.vd1[p] = a.vd0[o]; a.vd1[N + p] = a.vd0[N + o]; a.vd1[2 * N + p] = a.vd0[2 * N + o]; }
  a.id1[p] = myid;
  const float qv = a.qf0[o];
  a.qf1[p] = qv;
  if (a.qd0) a.qd1[p] = a.qd0[o];
  if (a.ty0) a.ty1[p] = a.ty0[o];
  a.im1[p] = a.im0[o];
  if (a.s4) a.s4[p] = make_uint4(sx, sy, sz, __float_as_uint(qv));
  if (mych) {
    a.cs[pc] = sx; a.cs[Nq + pc] = sy; a.cs[2 * Nq + pc] = sz;
    a.cqf[pc] = qv;
    if (a.cqd) a.cqd[pc] = a.qd0[o];
    a.cmap[pc] = (int32_t)p;
    if (a.cs4) a.cs4[pc] = make_uint4(sx, sy, sz, __float_as_uint(qv));
  }
}

constexpr int kCellsPerWarp = 4;

// One warp per kCellsPerWarp consecutive cells: rank members by their key (and charged
// members among themselves), then move every field to the final slot. When no cell of the four
// holds more than 8 (16) particles, each cell gets 8 (16) lanes; otherwise the warp takes the
// cells one after another, 32 members at a time.
__device__ __forceinline__ void bin_rank_permute_body(const PermuteArgs &a, int bx, int) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t c0 = (((int64_t)bx * blockDim.x + threadIdx.x) >> 5) * kCellsPerWarp;
  if (c0 >= a.ncell || gated_off(a.gate)) return;
  int cnt4 = 0;
  if (lane < kCellsPerWarp && c0 + lane < a.ncell)
    cnt4 = a.cell_start[c0 + lane + 1] - a.cell_start[c0 + lane];
  // Cells of at most 8 (16) members: 8-lane (16-lane) segments, one cell each, in one (two)
  // rounds; lanes past a cell's count hold the largest key. Larger cells: one cell after
  // another, 32 members at a time (below).
  const int mx = __reduce_max_sync(FULL, cnt4);
  if (mx <= 16) {
    const int W = mx <= 8 ? 8 : 16;
    const int lw = W == 8 ? 3 : 4;
    for (int r = 0; r < W / 8; ++r) {
      const int64_t c = c0 + r * (32 / W) + (lane >> lw);
      const int k = lane & (W - 1);
      const bool cell_ok = c < a.ncell;
      const int32_t beg = cell_ok ? a.cell_start[c] : 0;
      const int32_t cnt = cell_ok ? a.cell_start[c + 1] - beg : 0;
      const bool valid = k < cnt;
      const int32_t o = valid ? a.tmp[beg + k] : 0;
      const int32_t myid = valid ? a.id0[o] : INT_MAX;
      const uint64_t mykey = valid ? member_key(a, o, myid) : ~0ull;
      const int mych = (valid && a.qf0[o] != 0.0f) ? 1 : 0;
      int rank = 0, crank = 0;
      for (int t = 0; t < mx; ++t) {
        const uint64_t x = __shfl_sync(FULL, mykey, t, W);
        const int xc = __shfl_sync(FULL, mych, t, W);
        if (x < mykey) { ++rank; crank += xc; }
      }
      if (valid) move_particle(a, o, beg + rank, myid, mych != 0, a.ccell_start[c] + crank);
    }
    return;
  }
  for (int q = 0; q < kCellsPerWarp; ++q) {
    const int64_t c = c0 + q;
    if (c >= a.ncell) break;
    const int32_t beg = a.cell_start[c];
    const int32_t cnt = a.cell_start[c + 1] - beg;
    const int32_t cbeg = a.ccell_start[c];
    for (int kb = 0; kb < cnt; kb += 32) {
      const int k = kb + lane;
      const bool valid = k < cnt;
      const int32_t o = valid ? a.tmp[beg + k] : 0;
      const int32_t myid = valid ? a.id0[o] : INT_MAX;
      const uint64_t mykey = valid ? member_key(a, o, myid) : ~0ull;
      const bool mych = valid && a.qf0[o] != 0.0f;
      int rank = 0, crank = 0;
      for (int mb = 0; mb < cnt; mb += 32) {
        const int mm = mb + lane;
        const int32_t ov = mm < cnt ? a.tmp[beg + mm] : 0;
        const uint64_t okey = mm < cnt ? member_key(a, ov, a.id0[ov]) : ~0ull;
        const int och = (mm < cnt && a.qf0[ov] != 0.0f) ? 1 : 0;
        const int lim = min(32, cnt - mb);
        for (int t = 0; t < lim; ++t) {
          const uint64_t x = __shfl_sync(FULL, okey, t);
          const int xc = __shfl_sync(FULL, och, t);
          if (x < mykey) { ++rank; crank += xc; }
        }
      }
      if (valid) move_particle(a, o, beg + rank, myid, mych, cbeg + crank);
    }
  }
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), bin_rank_permute_kernel, PermuteArgs,
                   bin_rank_permute_body)

// Order kept (no list build this step): copy every field to the same slot of the other
// buffer and refresh the charged subset's coordinates through cmap. Threads [0, N) copy
// particles, threads [N, N + Nq) charged slots.
__device__ __forceinline__ void bin_identity_body(const PermuteArgs &a, int bx, int) {
  if (a.gate && *a.gate != 0) return;
  const int64_t k = (int64_t)bx * blockDim.x + threadIdx.x;
  const int64_t N = a.N, Nq = a.Nq;
  if (k < N) {
    const uint32_t sx = a.s0[k], sy = a.s0[N + k], sz = a.s0[2 * N + k];
    a.s1[k] = sx; a.s1[N + k] = sy; a.s1[2 * N + k] = sz;
    if (a.vf0) { a.vf1[k] = a.vf0[k]; a.vf1[N + k] = a.vf0[N + k]; a.vf1[2 * N + k] = a.vf0[2 * N + k]; }
    if (a.vd0) { a.vd1[k] = a.vd0[k]; a.vd1[N + k] = a.vd0[N + k]; a.vd1[2 * N + k] = a.vd0[2 * N + k]; }
    a.id1[k] = a.id0[k];
    const float qv = a.qf0[k];
    a.qf1[k] = qv;
    if (a.qd0) a.qd1[k] = a.qd0[k];
    if (a.ty0) a.ty1[k] = a.ty0[k];
    a.im1[k] = a.im0[k];
    if (a.s4) a.s4[k] = make_uint4(sx, sy, sz, __float_as_uint(qv));
  } else if (k < N + Nq) {
    const int64_t pc = k - N;
    const int64_t p = a.cmap[pc];
    const uint32_t sx = a.s0[p], sy = a.s0[N + p], sz = a.s0[2 * N + p];
    a.cs[pc] = sx; a.cs[Nq + pc] = sy; a.cs[2 * Nq + pc] = sz;
    if (a.cs4) a.cs4[pc] = make_uint4(sx, sy, sz, __float_as_uint(a.cqf[pc]));
  }
}
RBE_BATCHED_KERNEL(__launch_bounds__(256), bin_identity_kernel, PermuteArgs, bin_identity_body)

cudaError_t launch_bin_sort(Ctx &c) {
  const int64_t N = c.N, nc = c.grid.ncell;
  const int b0 = c.cur, b1 = 1 - c.cur;
  const int32_t *gate = c.vl_on ? c.vl_flags : nullptr;  // list mode: sort only on a build
  cudaError_t e = fill_zero(c, c.cell_count, 2 * nc);
  if (e != cudaSuccess) return e;
  if (N > 0) {
    const CountArgs a{N, c.s[b0], c.qf[b0], c.grid.n[0], c.grid.n[1], c.grid.n[2],
                      c.cell_count, c.ccell_count, c.key, c.off, gate};
    // (four particles a thread when N allows; a batch keeps one, so that replicas of any N
    //  share a class)
    if (N % 4 == 0 && !c.rec)
      e = dispatch(c, bin_count4_kernel, bin_count4_kernel_b,
                   dim3((unsigned)((N / 4 + 255) / 256)), dim3(256), 0, a);
    else
      e = dispatch(c, bin_count_kernel, bin_count_kernel_b, dim3((unsigned)((N + 255) / 256)),
                   dim3(256), 0, a);
    if (e != cudaSuccess) return e;
  }
  const int64_t nblk = c.scan_nblk;
  const ScanArgs sa{c.cell_count, c.cell_start, c.scan_blk, nc, nblk, gate};
  e = dispatch(c, scan_block_kernel, scan_block_kernel_b, dim3((unsigned)nblk, 2),
               dim3(kScanThreads), 0, sa);
  if (e != cudaSuccess) return e;
  e = dispatch(c, scan_top_kernel, scan_top_kernel_b, dim3(2), dim3(1024), 0, sa);
  if (e != cudaSuccess) return e;
  e = dispatch(c, scan_add_kernel, scan_add_kernel_b, dim3((unsigned)nblk, 2),
               dim3(kScanThreads), 0, sa);
  if (e != cudaSuccess) return e;
  if (N > 0) {
    const ScatterArgs xa{N, c.key, c.off, c.cell_start, c.tmp, gate};
    if (N % 4 == 0 && !c.rec)
      e = dispatch(c, bin_scatter4_kernel, bin_scatter4_kernel_b,
                   dim3((unsigned)((N / 4 + 255) / 256)), dim3(256), 0, xa);
    else
      e = dispatch(c, bin_scatter_kernel, bin_scatter_kernel_b, dim3((unsigned)((N + 255) / 256)),
                   dim3(256), 0, xa);
    if (e != cudaSuccess) return e;
    PermuteArgs a;
    a.N = N; a.Nq = c.Nq; a.ncell = nc;
    a.cell_start = c.cell_start; a.ccell_start = c.ccell_start; a.tmp = c.tmp;
    a.s0 = c.s[b0]; a.s1 = c.s[b1];
    a.vf0 = c.vf[b0]; a.vf1 = c.vf[b1];
    a.vd0 = c.vd[b0]; a.vd1 = c.vd[b1];
    a.id0 = c.id[b0]; a.id1 = c.id[b1];
    a.qf0 = c.qf[b0]; a.qf1 = c.qf[b1];
    a.qd0 = c.qd[b0]; a.qd1 = c.qd[b1];
    a.ty0 = c.type[b0]; a.ty1 = c.type[b1];
    a.im0 = c.invm[b0]; a.im1 = c.invm[b1];
    a.cs = c.cs; a.cqf = c.cqf; a.cqd = c.cqd; a.cmap = c.cmap;
    a.s4 = c.vl_on ? c.s4 : nullptr;  // the list gathers
    a.cs4 = c.vl_on ? c.cs4 : c.cq4;  // list gathers, or the Coulomb pass
    a.gate = gate;
    const int64_t threads = (nc + kCellsPerWarp - 1) / kCellsPerWarp * 32;
    e = dispatch(c, bin_rank_permute_kernel, bin_rank_permute_kernel_b, dim3((unsigned)((threads + 255) / 256)), dim3(256), 0, a);
    if (e != cudaSuccess) return e;
    if (gate) {
      e = dispatch(c, bin_identity_kernel, bin_identity_kernel_b, dim3((unsigned)((N + c.Nq + 255) / 256)), dim3(256), 0, a);
      if (e != cudaSuccess) return e;
    }
  }
  c.cur = b1;
  return cudaGetLastError();
}

}  // namespace rbe
