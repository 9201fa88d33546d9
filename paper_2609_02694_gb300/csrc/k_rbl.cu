// k_rbl.cu -- random batch list short-range force (Eqs. Ci_Si, RBL, F_corr).
//
// For each particle i, with cells of side >= r_s:
//   C_i = {j != i: r_ij <= r_core}, S_i = {j: r_core < r_ij <= r_s}
//   F~_i = sum_{C_i} F_ij + (#S_i / p) sum_{B_i} F_ij,  B_i = p i.i.d. uniform draws from S_i
//   F_i  = F~_i - (1/N) sum_j F~_j
// (The paper's core cutoff r_c is `r_core` here and its r_s is the real-space cutoff.)
// S_i is enumerated in a canonical order shared with the oracle: the 27 neighbour cells
// in (dz, dy, dx) order, each offset from -1 to 1, and inside each cell the (s_x, id)
// order of the binning. Draw t takes idx = floor(w * #S_i / 2^32), where w is word
// (t mod 4) of Philox4x32-10 with counter (id_i, t / 4, step, 1). When #S_i <= p the whole
// shell enters with weight 1.
//
// Work decomposition: one thread per i. Lanes of a warp whose cells share a row (c_y, c_z)
// and lie within `gs` cells in x form a group; gs > 1 only in dilute systems, so that a
// group fills the warp. The group walks the union of its members' 27-cell stencils: the
// 9 rows (dz, dy) in canonical order, each a run of gs + 2 cells in x. Every candidate
// carries its x offset in that run, and a lane keeps only candidates of its own three x
// cells; in canonical order these form exactly the lane's own S_i order. Candidates are
// staged in shared memory in FP32 coordinates relative to the group leader. Membership is
// decided exactly: FP32 outside a band around r_core^2 and r_s^2 (+-1e-5, or the FP32
// error bound of the group's extent where that is larger), the FP64 oracle expression
// inside it.
// Cells keep their members in (s_x, id) order, so each row's run is sorted by x and is cut
// to the x-range some member of the group can reach (binary searches on exact unwrapped
// coordinates); trimmed candidates are beyond r_s of every member.
// Pass 1 classifies every candidate once in canonical order, evaluates the core pairs from
// the staged exact integer displacements (branch-light), and keeps per lane the shell
// members of each 32-candidate chunk: their count in shared memory and their bit mask in a
// per-warp scratch row in global memory. Pass 2 draws, sorts the draws, finds each draw's
// chunk from the counts and its candidate from the mask (n-th set bit), and evaluates the
// drawn pairs: no candidate is classified twice.
// The scratch is sized by the blocks that can be resident at once, not by N: each block
// takes a free slot of a pool with one slot per block the GPU can hold (numbered by
// compare-and-swap probes that always succeed, since at most that many blocks are resident)
// and frees it when it ends.
// Eager variant, for shells that are mostly no larger than p (dilute systems): pass 1 also
// evaluates every shell pair, in canonical order, into a second accumulator; each lane
// queues its chunks' pair masks and a window of four chunks is evaluated with one uniform
// trip count (its heaviest lane). A particle
// with #S_i <= p then keeps it (the same sum pass 2 would form, bit for bit) and skips
// pass 2; one with #S_i > p discards it and draws as above.
// The mean-force correction is a fixed-order FP64 reduction followed by a subtraction.
#include <algorithm>
#include <climits>
#include <cmath>

#include "pair_common.cuh"

namespace rbe {

constexpr int kRblWarps = 1;  // one warp a block: no warp waits for a slower one
constexpr int kRblMaxP = 32;
constexpr int kRblWin = 4;          // chunks of 32 candidates per window
constexpr int kRblMaxChunks = 192;  // candidates per group <= 6144
constexpr int kRblMaxSpan = 14;     // x cells per group (gs)

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
  int *err;
  int gs;  // group extent in x cells (1 .. kRblMaxSpan, gs + 2 <= n_x)
  uint32_t *masks;  // per slot and warp: kRblMaxChunks x 32 shell masks
  int *slots;       // slot pool (0 free, 1 taken)
  int nslots;
};

// x offset of cell cxj in the group's run of cells gx - 1 .. gx + gs (mod n_x)
__device__ __forceinline__ int run_offset(int cxj, int gx, int n0) {
  int d = cxj - gx + 1;  // in [-(n0 - 2), n0]
  d += d < 0 ? n0 : 0;
  d -= d >= n0 ? n0 : 0;
  return d;
}

// Coarse FP32 classes with the exact FP64 decision inside the bands of r_core^2 and r_s^2
// (at least +-1e-5, wider for long groups): 0 outside, 1 core (r <= r_core), 2 shell
// (r_core < r <= r_s).
__device__ __forceinline__ int rbl_class(const RblArgs &a, float r2, int dsx, int dsy, int dsz) {
  if (r2 < a.rcore2_lo) return 1;
  if (r2 > a.rs2_hi) return 0;
  if (r2 > a.rcore2_hi && r2 < a.rs2_lo) return 2;
  const double e2 = exact_r2(a.pa.pc, dsx, dsy, dsz);
  if (e2 <= a.rcore2d) return 1;
  if (e2 <= a.rs2d) return 2;
  return 0;
}

template <typename real, bool COUL, bool MULTI>
__device__ __forceinline__ void rbl_pair_ds(const RblArgs &a, const LJTable *tab, int dsx,
                                            int dsy, int dsz, real qi, int ti, real qj, int tj,
                                            PairAcc<real> &acc) {
  const PairConst &pc = a.pa.pc;
  real dx, dy, dz;
  if (sizeof(real) == 8) {
    dx = (real)((double)dsx * pc.hd[0]); dy = (real)((double)dsy * pc.hd[1]); dz = (real)((double)dsz * pc.hd[2]);
  } else {
    dx = (real)((float)dsx * pc.h[0]); dy = (real)((float)dsy * pc.h[1]); dz = (real)((float)dsz * pc.h[2]);
  }
  const real r2 = mad(dx, dx, mad(dy, dy, dz * dz));
  pair_force_v<real, true, COUL, MULTI>(a.pa, tab, dx, dy, dz, r2, qi, ti, qj, tj, acc);
}

// One pair with a 0/1 activity mask (idle lanes compute a finite dummy with q_j = 0).
template <typename real, bool COUL, bool MULTI>
__device__ __forceinline__ PairAcc<real> rbl_pair_eval(const RblArgs &a, const LJTable *tab, bool act,
                                                       int dsx, int dsy, int dsz, real qi, int ti,
                                                       real qj, int tj) {
  const PairConst &pc = a.pa.pc;
  real dx, dy, dz;
  if (sizeof(real) == 8) {
    dx = (real)((double)dsx * pc.hd[0]); dy = (real)((double)dsy * pc.hd[1]); dz = (real)((double)dsz * pc.hd[2]);
  } else {
    dx = (real)((float)dsx * pc.h[0]); dy = (real)((float)dsy * pc.h[1]); dz = (real)((float)dsz * pc.h[2]);
  }
  const real r2 = mad(dx, dx, mad(dy, dy, dz * dz));
  const real on = act ? (real)1 : (real)0;
  const real r2s = act ? r2 : (real)1;
  PairAcc<real> t;
  t.fx = t.fy = t.fz = t.ulj = t.wlj = t.uc = t.wc = t.cuc = t.cwc = (real)0;
  t.nbr = 0;
  pair_force_v<real, true, COUL, MULTI>(a.pa, tab, dx * on, dy * on, dz * on, r2s, qi, ti,
                                        act ? qj : (real)0, tj, t);
  return t;
}

// acc += t where `on`, unchanged bit for bit otherwise.
template <typename real>
__device__ __forceinline__ void rbl_acc_add(const RblArgs &a, bool on_, const PairAcc<real> &t,
                                            PairAcc<real> &acc) {
  const real on = on_ ? (real)1 : (real)0;
  acc.fx = mad(on, t.fx, acc.fx); acc.fy = mad(on, t.fy, acc.fy); acc.fz = mad(on, t.fz, acc.fz);
  acc.ulj = mad(on, t.ulj, acc.ulj); acc.wlj = mad(on, t.wlj, acc.wlj);
  if (a.pa.comp) {
    real s = acc.uc, cs = acc.cuc, w = acc.wc, cw = acc.cwc;
    kahan_add(s, cs, t.uc);
    kahan_add(w, cw, t.wc);
    acc.uc = on_ ? s : acc.uc; acc.cuc = on_ ? cs : acc.cuc;
    acc.wc = on_ ? w : acc.wc; acc.cwc = on_ ? cw : acc.cwc;
  } else {
    acc.uc = mad(on, t.uc, acc.uc);
    acc.wc = mad(on, t.wc, acc.wc);
  }
}

// 16 one-warp blocks per SM (at most 128 registers): the compiler's own choice spilled in
// the eager variant.
template <typename real, bool COUL, bool MULTI, bool WRAP, bool EAGER>
__global__ void __launch_bounds__(kRblWarps * 32, 16) rbl_kernel(const RblArgs a) {
  __shared__ float4 stage[kRblWarps][kRblWin][32];
  __shared__ int4 stage_d[kRblWarps][kRblWin][32];
  __shared__ float stage_q[kRblWarps][kRblWin][32];
  __shared__ int32_t stage_j[kRblWarps][kRblWin][32];
  __shared__ int32_t seg_beg[kRblWarps][18];
  __shared__ int32_t seg_pre[kRblWarps][19];
  __shared__ uint32_t tmask[kRblWarps][kRblWin][kRblMaxSpan + 2];  // candidates per x offset
  __shared__ uint8_t ccount[kRblWarps][kRblMaxChunks][32];  // shell members per chunk, per lane
  // per lane, the window's chunks with pairs to evaluate: (eval mask, core mask) and chunk
  __shared__ uint2 rq[kRblWarps][kRblWin][32];
  __shared__ uint8_t rqw[kRblWarps][kRblWin][32];
  __shared__ double wred[kRblWarps][NQ_PAIR + 3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  __shared__ int slot_s;
  const PairSet &S = a.pa.set;
  const int64_t n = S.n;
  const LJTable *tab = a.pa.table;
  if (threadIdx.x == 0) {  // a free scratch slot (at most nslots blocks are resident)
    int got = -1;
    for (int k = 0; k < a.nslots && got < 0; ++k) {
      const int sl = (int)((blockIdx.x + (unsigned)k) % (unsigned)a.nslots);
      if (atomicCAS(&a.slots[sl], 0, 1) == 0) got = sl;
    }
    if (got < 0) atomicOr(a.err, ERRBIT_CAPACITY);
    // acquire: the previous owner released the slot after a device-scope fence, so its
    // stores to the slot's rows are ordered before every access of this block
    __threadfence();
    slot_s = got;
  }
  __syncthreads();
  const int slot = slot_s;
  uint32_t *const scr =
      a.masks + ((int64_t)(slot < 0 ? 0 : slot) * kRblWarps + wid) * (int64_t)kRblMaxChunks * 32;
  const int64_t i0 = ((int64_t)blockIdx.x * kRblWarps + wid) * 32;
  const int64_t i = i0 + lane;
  const bool valid = i < n && slot >= 0;
  // shell: the drawn shell pairs; in the eager variant first every shell pair, reset when
  // the particle turns out to need draws
  PairAcc<real> core, shell;
  core.fx = core.fy = core.fz = core.ulj = core.wlj = core.uc = core.wc = (real)0;
  core.cuc = core.cwc = (real)0;
  core.nbr = 0;
  shell = core;
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
    int ncore = 0, nsh = 0, ksh = 0;
    unsigned remaining = __ballot_sync(FULL, valid);
    while (remaining) {
      const int leader = __ffs(remaining) - 1;
      const int gx = __shfl_sync(FULL, cx, leader), gy = __shfl_sync(FULL, cy, leader),
                gz = __shfl_sync(FULL, cz, leader);
      const bool in = valid && cy == gy && cz == gz && (unsigned)(cx - gx) < (unsigned)a.gs;
      remaining &= ~__ballot_sync(FULL, in);
      const int lo = cx - gx;  // the lane's x cells are offsets lo .. lo + 2 of the run
      const uint32_t ox = __shfl_sync(FULL, sxi, leader), oy = __shfl_sync(FULL, syi, leader),
                     oz = __shfl_sync(FULL, szi, leader);
      const int dxi = (int)(sxi - ox), dyi = (int)(syi - oy), dzi = (int)(szi - oz);
      const float xi = __fmul_rn((float)dxi, a.pa.pc.h[0]);
      const float yi = __fmul_rn((float)dyi, a.pa.pc.h[1]);
      const float zi = __fmul_rn((float)dzi, a.pa.pc.h[2]);
      // The 9 rows (dz, dy) in canonical order, each the x cells gx - 1 .. gx + gs (mod n_x)
      // as at most two contiguous runs; one lane per run. Every row of cells is sorted by x,
      // so each run is cut to the x-range some member can reach: members span [gxlo, gxhi]
      // in x, and a row whose cells lie at y/z distance d from the group's box reaches only
      // sqrt(r_s^2 - d^2) in x. The cut searches exact unwrapped coordinates (s_x plus the
      // run's wrap shift), which are monotone along a run; trimmed candidates are beyond r_s
      // of every member, so the canonical shell order of each lane is unchanged.
      const int gxlo = __reduce_min_sync(FULL, in ? dxi : INT_MAX);
      const int gxhi = __reduce_max_sync(FULL, in ? dxi : INT_MIN);
      const int gylo = __reduce_min_sync(FULL, in ? dyi : INT_MAX);
      const int gyhi = __reduce_max_sync(FULL, in ? dyi : INT_MIN);
      const int gzlo = __reduce_min_sync(FULL, in ? dzi : INT_MAX);
      const int gzhi = __reduce_max_sync(FULL, in ? dzi : INT_MIN);
      {
        int b0 = 0, l0 = 0;
        if (lane < 18) {
          const int r = lane >> 1, part = lane & 1;
          const int dz = r / 3 - 1, dy = r % 3 - 1;
          const int ry = ((gy + dy) % n1 + n1) % n1, rz = ((gz + dz) % n2 + n2) % n2;
          const int64_t rowbase = (int64_t)n0 * (ry + (int64_t)n1 * rz);
          const int xlo = gx - 1, xhi = gx + a.gs;
          int c0, c1;  // inclusive cell range of this run (empty when c1 < c0)
          if (xlo < 0) { c0 = part ? 0 : n0 - 1; c1 = part ? xhi : n0 - 1; }
          else if (xhi >= n0) { c0 = part ? 0 : xlo; c1 = part ? xhi - n0 : n0 - 1; }
          else { c0 = xlo; c1 = part ? xlo - 1 : xhi; }
          if (c1 >= c0) {
            b0 = S.cell_start[rowbase + c0];
            l0 = S.cell_start[rowbase + c1 + 1] - b0;
          }
          if (!WRAP && l0 > 0) {
            // row extent in frame units (cells gy + dy, gz + dz unwrapped, edges rounded
            // outward by 2 units), distance from the group's box, x-reach (radius widened by
            // 1e-9, rounded up, +2 units)
            const double wy = 4294967296.0 / n1, wz = 4294967296.0 / n2;
            const double ylo = (gy + dy) * wy - (double)oy - 2.0, yhi = (gy + dy + 1) * wy - (double)oy + 2.0;
            const double zlo = (gz + dz) * wz - (double)oz - 2.0, zhi = (gz + dz + 1) * wz - (double)oz + 2.0;
            const double ddy = fmax(0.0, fmax(ylo - gyhi, gylo - yhi)) * a.pa.pc.hd[1];
            const double ddz = fmax(0.0, fmax(zlo - gzhi, gzlo - zhi)) * a.pa.pc.hd[2];
            const double rx2 = a.pa.pc.rc2d * (1.0 + 1e-9) - ddy * ddy - ddz * ddz;
            if (rx2 <= 0.0) {
              l0 = 0;
            } else {
              const int64_t rx = (int64_t)(ceil(sqrt(rx2) / a.pa.pc.hd[0]) + 2.0);
              // the part left of x = 0 (cell n_x - 1 standing for -1) or right of x = L
              const int64_t sh = (xlo < 0 && !part) ? -((int64_t)1 << 32)
                                 : (xhi >= n0 && part) ? ((int64_t)1 << 32) : 0;
              auto first_ge = [&](int64_t key) {
                int lo_ = 0, hi_ = l0;
                while (lo_ < hi_) {
                  const int mid = (lo_ + hi_) >> 1;
                  if ((int64_t)S.sx[b0 + mid] + sh - (int64_t)ox < key) lo_ = mid + 1;
                  else hi_ = mid;
                }
                return lo_;
              };
              const int u = first_ge((int64_t)gxlo - rx), v = first_ge((int64_t)gxhi + rx + 1);
              b0 += u;
              l0 = v - u;
            }
          }
        }
        int incl = l0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += v;
        }
        if (lane < 18) {
          seg_beg[wid][lane] = b0;
          seg_pre[wid][lane] = incl - l0;
        }
        if (lane == 17) seg_pre[wid][18] = incl;
      }
      __syncwarp();
      const int T = seg_pre[wid][18];
      const int nchunks = (T + 31) / 32;
      if (nchunks > kRblMaxChunks) {  // capacity of the per-lane chunk counts
        if (lane == 0) atomicOr(a.err, ERRBIT_CAPACITY);
        continue;
      }
      // ---- pass 1: classify every candidate in canonical order, evaluate the core pairs,
      //      keep the number of shell members of each 32-candidate chunk
      int sg = 0;
      for (int base = 0; base < T; base += 32 * kRblWin) {
        // (window loops stay rolled: the unrolled kernel outgrew the instruction cache)
#pragma unroll 1
        for (int w = 0; w < kRblWin; ++w) {
          const int c = base + 32 * w + lane;
          int s = sg, tc = -1;
          if (c < T) {
            while (seg_pre[wid][s + 1] <= c) ++s;
            const int64_t j = seg_beg[wid][s] + (c - seg_pre[wid][s]);
            const uint32_t sxj = S.sx[j];
            const int dxj = (int)(sxj - ox), dyj = (int)(S.sy[j] - oy), dzj = (int)(S.sz[j] - oz);
            if (a.gs > 1) tc = run_offset(cell_of(sxj, n0), gx, n0);  // x offset in the run
            // products rounded explicitly (no contraction): the classification is a fixed
            // function of the integer coordinates
            stage[wid][w][lane] = make_float4(__fmul_rn((float)dxj, a.pa.pc.h[0]),
                                              __fmul_rn((float)dyj, a.pa.pc.h[1]),
                                              __fmul_rn((float)dzj, a.pa.pc.h[2]), 0.f);
            stage_d[wid][w][lane] = make_int4(dxj, dyj, dzj, MULTI ? S.type[j] : 0);
            if (COUL) stage_q[wid][w][lane] = S.qf[j];
            stage_j[wid][w][lane] = (int32_t)j;
          }
          if (a.gs > 1)  // (one-cell groups keep every candidate)
            for (int t = 0; t < a.gs + 2; ++t) {
              const uint32_t mt = __ballot_sync(FULL, tc == t);
              if (lane == 0) tmask[wid][w][t] = mt;
            }
          sg = __shfl_sync(FULL, s, 31);
        }
        __syncwarp();
        int nq = 0, qcnt = 0;  // eager: queued chunks and pairs of this lane in the window
#pragma unroll 1
        for (int w = 0; w < kRblWin; ++w) {
          const int nj = max(0, min(32, T - base - 32 * w));
          uint32_t mcore = 0u, mshell = 0u, mamb = 0u;
          if (nj > 0) {
            // Four threshold tests per candidate, each the sign bit of a difference shifted
            // into a mask (one funnel shift; the sign of a rounded difference is exact):
            // lo1 = r2 < rcore2_lo, up1 = r2 > rcore2_hi, lo2 = r2 < rs2_lo, up2 = r2 > rs2_hi.
            // Candidate tt lands in bit 31 - tt; the masks are bit-reversed afterwards.
            uint32_t lo1 = 0u, up1 = 0u, lo2 = 0u, up2 = 0u;
#pragma unroll
            for (int tt = 0; tt < 32; ++tt) {
              const float4 pj = stage[wid][w][tt];
              float ddx = xi - pj.x, ddy = yi - pj.y, ddz = zi - pj.z;
              if (WRAP) {
                ddx = fold(ddx, a.pa.L[0], a.pa.invL[0]);
                ddy = fold(ddy, a.pa.L[1], a.pa.invL[1]);
                ddz = fold(ddz, a.pa.L[2], a.pa.invL[2]);
              }
              const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
              lo1 = __funnelshift_l(__float_as_uint(r2 - a.rcore2_lo), lo1, 1);
              up1 = __funnelshift_l(__float_as_uint(a.rcore2_hi - r2), up1, 1);
              lo2 = __funnelshift_l(__float_as_uint(r2 - a.rs2_lo), lo2, 1);
              up2 = __funnelshift_l(__float_as_uint(a.rs2_hi - r2), up2, 1);
            }
            lo1 = __brev(lo1); up1 = __brev(up1); lo2 = __brev(lo2); up2 = __brev(up2);
            mcore = lo1;                                   // r2 < rcore2_lo
            mshell = up1 & lo2;                            // rcore2_hi < r2 < rs2_lo
            mamb = (~lo1 & ~up1) | (~lo2 & ~up2);          // inside one of the two bands
            uint32_t vmask = nj >= 32 ? 0xFFFFFFFFu : ((1u << nj) - 1u);
            if (!in) vmask = 0u;
            else if (a.gs > 1) vmask &= tmask[wid][w][lo] | tmask[wid][w][lo + 1] | tmask[wid][w][lo + 2];
            mcore &= vmask; mshell &= vmask; mamb &= vmask;
            while (mamb) {  // rare: exact decision inside the bands
              const int tt = __ffs(mamb) - 1;
              mamb &= mamb - 1u;
              const int4 d = stage_d[wid][w][tt];
              const int cls = rbl_class(a, a.rs2_hi, (int)((uint32_t)dxi - (uint32_t)d.x),
                                        (int)((uint32_t)dyi - (uint32_t)d.y),
                                        (int)((uint32_t)dzi - (uint32_t)d.z));
              if (cls == 1) mcore |= 1u << tt;
              if (cls == 2) mshell |= 1u << tt;
            }
          }
          const int chunk = (base >> 5) + w;
          if (chunk < nchunks) {
            ccount[wid][chunk][lane] = (uint8_t)__popc(mshell);
            scr[chunk * 32 + lane] = mshell;  // coalesced, read back by pass 2
          }
          nsh += __popc(mshell);
          if (EAGER) {  // core and shell pairs are evaluated per window below
            const uint32_t bits = mcore | mshell;
            if (bits != 0u) {
              rq[wid][nq][lane] = make_uint2(bits, mcore);
              rqw[wid][nq][lane] = (uint8_t)w;
              ++nq;
            }
            qcnt += __popc(bits);
            continue;
          }
          // core pairs, branch-light, in canonical order, one uniform trip count per chunk
          // (a few core pairs per chunk and lane); the particle itself (r = 0) is skipped
          uint32_t bits = mcore;
          const int nbits = __reduce_max_sync(FULL, __popc(bits));
          for (int kb = 0; kb < nbits; ++kb) {
            const bool act = bits != 0u;
            const int tt = act ? __ffs(bits) - 1 : 0;
            bits &= bits - 1u;
            const int32_t j = stage_j[wid][w][tt];
            const bool use = act && j != (int32_t)i;
            const int4 d = stage_d[wid][w][tt];
            real qj = (real)0;
            if (COUL) qj = sizeof(real) == 8 ? (use ? (real)S.qd[j] : (real)0) : (real)stage_q[wid][w][tt];
            ncore += use ? 1 : 0;
            const PairAcc<real> t = rbl_pair_eval<real, COUL, MULTI>(
                a, tab, use, (int)((uint32_t)dxi - (uint32_t)d.x), (int)((uint32_t)dyi - (uint32_t)d.y),
                (int)((uint32_t)dzi - (uint32_t)d.z), qi, ti, qj, d.w);
            rbl_acc_add(a, use, t, core);
          }
        }
        // Eager: the window's core and shell pairs, branch-light, each lane in canonical
        // order, with one uniform trip count for the window (the lane with the most pairs)
        // instead of one per chunk; the particle itself (r = 0, always core) is skipped.
        if (EAGER) {
          const int nit = __reduce_max_sync(FULL, qcnt);
          int hq = 0, cw = 0;
          uint32_t cm = 0u, cc = 0u;  // the chunk being consumed: pairs left, core pairs
          for (int kb = 0; kb < nit; ++kb) {
            const bool act = kb < qcnt;
            const uint2 e = rq[wid][hq & (kRblWin - 1)][lane];
            const int ew = rqw[wid][hq & (kRblWin - 1)][lane];
            const bool take = act && cm == 0u;
            cm = take ? e.x : cm;
            cc = take ? e.y : cc;
            cw = take ? ew : cw;
            hq += take ? 1 : 0;
            const int tt = act ? __ffs(cm) - 1 : 0;
            const int w = act ? cw : 0;  // (idle lanes: candidate 0 of chunk 0, staged)
            cm &= cm - 1u;
            const int32_t j = stage_j[wid][w][tt];
            const bool use = act && j != (int32_t)i;
            const bool is_core = ((cc >> tt) & 1u) != 0u;
            const int4 d = stage_d[wid][w][tt];
            real qj = (real)0;
            if (COUL) qj = sizeof(real) == 8 ? (use ? (real)S.qd[j] : (real)0) : (real)stage_q[wid][w][tt];
            ncore += (use && is_core) ? 1 : 0;
            const PairAcc<real> t = rbl_pair_eval<real, COUL, MULTI>(
                a, tab, use, (int)((uint32_t)dxi - (uint32_t)d.x), (int)((uint32_t)dyi - (uint32_t)d.y),
                (int)((uint32_t)dzi - (uint32_t)d.z), qi, ti, qj, d.w);
            rbl_acc_add(a, use && is_core, t, core);
            if (EAGER) {
              rbl_acc_add(a, use && !is_core, t, shell);
              if (a.partners && use && !is_core) {  // shell rank ksh in canonical order
                if (ksh < a.p) a.partners[i * a.p + ksh] = a.id[j];
                ++ksh;
              }
            }
          }
        }
        __syncwarp();
      }
      // ---- pass 2: the drawn shell partners (all of them when #S_i <= p; the eager
      //      variant has that sum, and the partners, already and runs pass 2 only to draw)
      const bool pass2 = in && (!EAGER || nsh > a.p);
      if (EAGER && in && !pass2 && a.partners)
        for (int t = nsh; t < a.p; ++t) a.partners[i * a.p + t] = -1;
      if (EAGER && pass2) {  // the eager sum is not the estimator here: draw instead
        shell.fx = shell.fy = shell.fz = shell.ulj = shell.wlj = shell.uc = shell.wc = (real)0;
        shell.cuc = shell.cwc = (real)0;
      }
      if (pass2) {
        uint32_t idx[kRblMaxP];
        int ord[kRblMaxP];
        int ndraw;
        if (a.partners)
          for (int t = 0; t < a.p; ++t) a.partners[i * a.p + t] = -1;
        if (nsh > a.p) {
          const uint32_t st = (uint32_t)(*a.step);
          for (int t = 0; t < a.p; t += 4) {
            const uint4 w4 = philox4x32_10(make_uint4(idi, (uint32_t)(t / 4), st, 1u), a.key);
            const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
            for (int u = 0; u < 4 && t + u < a.p; ++u)
              idx[t + u] = (uint32_t)(((uint64_t)ww[u] * (uint64_t)nsh) >> 32);
          }
          ndraw = a.p;
          for (int t = 0; t < ndraw; ++t) ord[t] = t;
          for (int t = 1; t < ndraw; ++t) {  // insertion sort by index, stable in t
            const int v = ord[t];
            int u = t - 1;
            while (u >= 0 && idx[ord[u]] > idx[v]) { ord[u + 1] = ord[u]; --u; }
            ord[u + 1] = v;
          }
        } else {
          ndraw = nsh;
          for (int t = 0; t < ndraw; ++t) { idx[t] = (uint32_t)t; ord[t] = t; }
        }
        // draws in canonical order: chunk from the counts, candidate from the chunk's mask
        int chunk = 0, before = 0, sgd = 0;
        for (int ptr = 0; ptr < ndraw; ++ptr) {
          const int target = (int)idx[ord[ptr]];
          while (before + (int)ccount[wid][chunk][lane] <= target) {
            before += ccount[wid][chunk][lane];
            ++chunk;
          }
          const uint32_t mk = scr[chunk * 32 + lane];
          const uint32_t pos = __fns(mk, 0u, target - before + 1);
          if (pos > 31u) {  // counts and masks disagree: cannot happen; never index with it
            atomicOr(a.err, ERRBIT_CAPACITY);
            continue;
          }
          const int c = chunk * 32 + (int)pos;
          while (seg_pre[wid][sgd + 1] <= c) ++sgd;  // draws ascend, so runs do too
          const int64_t j = seg_beg[wid][sgd] + (c - seg_pre[wid][sgd]);
          const int dsx = (int)((uint32_t)dxi - (S.sx[j] - ox));
          const int dsy = (int)((uint32_t)dyi - (S.sy[j] - oy));
          const int dsz = (int)((uint32_t)dzi - (S.sz[j] - oz));
          real qj = (real)0;
          if (COUL) qj = sizeof(real) == 8 ? (real)S.qd[j] : (real)S.qf[j];
          const PairAcc<real> t = rbl_pair_eval<real, COUL, MULTI>(
              a, tab, true, dsx, dsy, dsz, qi, ti, qj, MULTI ? S.type[j] : 0);
          rbl_acc_add(a, true, t, shell);
          if (a.partners) a.partners[i * a.p + ord[ptr]] = a.id[j];
        }
      }
    }
    if (valid) {
      const real w = nsh > a.p ? (real)nsh / (real)a.p : (real)1;
      fx = mad(w, shell.fx, core.fx);
      fy = mad(w, shell.fy, core.fy);
      fz = mad(w, shell.fz, core.fz);
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
  // release, after the block's last use of its rows (every warp is past the barrier above):
  // the fence orders all of the block's row stores before the flag store that frees the slot
  if (threadIdx.x == 0 && slot >= 0) {
    __threadfence();
    atomicExch(&a.slots[slot], 0);
  }
}

// The RBL kernel leaves one partial per block (energies, virials: NQ_PAIR doubles; sum of
// F~: 3 doubles). This pass sums fixed contiguous ranges of them into `ncomp` partials, in a
// fixed order, so the totals and the mean below read few slots whatever N is.
__global__ void __launch_bounds__(256) rbl_compact_kernel(const double *__restrict__ epart,
                                                          const double *__restrict__ fpart,
                                                          int64_t nblk, int64_t per,
                                                          double *__restrict__ eout,
                                                          double *__restrict__ fout) {
  constexpr int NV = NQ_PAIR + 3;
  __shared__ double sh[NV][256];
  const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(nblk, b0 + per);
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NQ_PAIR; ++k) acc[k] += epart[b * NQ_PAIR + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[NQ_PAIR + k] += fpart[b * 3 + k];
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < NQ_PAIR) eout[(int64_t)blockIdx.x * NQ_PAIR + threadIdx.x] = sh[threadIdx.x][0];
  else if (threadIdx.x < NV) fout[(int64_t)blockIdx.x * 3 + threadIdx.x - NQ_PAIR] = sh[threadIdx.x][0];
}

int64_t rbl_compact_count(int64_t nblk) { return std::max<int64_t>(1, std::min<int64_t>(nblk, 1024)); }

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

template <typename real, bool COUL, bool EAGER>
static void rbl_launch(const RblArgs &a, int64_t blocks, bool multi, bool wrap, cudaStream_t st) {
  const dim3 g((unsigned)blocks), b(kRblWarps * 32);
  if (wrap) {
    if (multi) rbl_kernel<real, COUL, true, true, EAGER><<<g, b, 0, st>>>(a);
    else rbl_kernel<real, COUL, false, true, EAGER><<<g, b, 0, st>>>(a);
  } else {
    if (multi) rbl_kernel<real, COUL, true, false, EAGER><<<g, b, 0, st>>>(a);
    else rbl_kernel<real, COUL, false, false, EAGER><<<g, b, 0, st>>>(a);
  }
}

template <typename real>
static void rbl_launch(const RblArgs &a, int64_t blocks, bool coul, bool eager, bool multi,
                       bool wrap, cudaStream_t st) {
  if (coul) {
    if (eager) rbl_launch<real, true, true>(a, blocks, multi, wrap, st);
    else rbl_launch<real, true, false>(a, blocks, multi, wrap, st);
  } else {
    if (eager) rbl_launch<real, false, true>(a, blocks, multi, wrap, st);
    else rbl_launch<real, false, false>(a, blocks, multi, wrap, st);
  }
}

// Group extent gs in x cells (enough cells to fill a warp: 1 unless the system is dilute,
// unless set by RBE_TUNE_RBL_SPAN; gs + 2 <= n_x keeps the union's cells distinct) and
// whether the leader frame needs the wrapping variant.
static void rbl_shape(const Ctx &c, int *gs_out, bool *wrap_out) {
  int gs = c.rbl_span;
  if (gs <= 0) {
    const double per_cell = (double)c.N / (double)c.grid.ncell;
    gs = per_cell > 0.0 ? (int)std::floor(32.0 / per_cell) : 1;
  }
  gs = std::max(1, std::min(std::min(gs, kRblMaxSpan), c.grid.n[0] - 2));
  // the leader frame is a valid minimum image while (group extent) + r_s < L/2
  bool wrap = false;
  for (int d = 0; d < 3; ++d)
    if (!(c.box[d] / c.grid.n[d] + c.rc < 0.5 * c.box[d] * (1.0 - 1e-9))) wrap = true;
  if (!wrap)
    while (gs > 1 && !(gs * c.box[0] / c.grid.n[0] + c.rc < 0.5 * c.box[0] * (1.0 - 1e-9))) --gs;
  *gs_out = gs;
  *wrap_out = wrap;
}

// Slots of the scratch pool: the most 128-thread blocks the GPU can hold at once (thread
// limit per SM), never more than the grid has blocks.
int64_t rbl_slot_count(int64_t n, int sms) {
  int dev = 0, thr = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      thr < 1) {
    cudaGetLastError();
    thr = 2048;  // the largest per-SM thread count of current GPUs: an upper bound on residency
  }
  const int64_t per_sm = std::max(1, thr / (kRblWarps * 32));
  return std::max<int64_t>(1, std::min<int64_t>(rbl_blocks(n), (int64_t)sms * per_sm));
}

int64_t rbl_mask_words(int64_t slots) { return slots * kRblWarps * (int64_t)kRblMaxChunks * 32; }

cudaError_t launch_rbl(Ctx &c, bool want_debug) {
  const int b = c.cur;
  RblArgs a;
  PairArgs &pa = a.pa;
  pa.grid = c.grid;
  pa.pc = c.pc;
  pa.ljA = c.lj.A[0]; pa.ljB = c.lj.B[0]; pa.ljA12 = c.lj.A12[0]; pa.ljB6 = c.lj.B6[0];
  pa.ljAd = c.lj.Ad[0]; pa.ljBd = c.lj.Bd[0]; pa.ljA12d = c.lj.A12d[0]; pa.ljB6d = c.lj.B6d[0];
  pa.table = reinterpret_cast<const LJTable *>(c.lj_dev);
  pa.F = c.F; pa.Fd = c.Fd; pa.Fstride = c.N; pa.accumulate = 0;
  pa.set.sx = c.s[b]; pa.set.sy = c.s[b] + c.N; pa.set.sz = c.s[b] + 2 * c.N;
  pa.set.qf = c.qf[b]; pa.set.qd = c.qd[b]; pa.set.type = c.type[b];
  pa.set.cell_start = c.cell_start; pa.set.map = nullptr; pa.set.n = c.N;
  pa.epart = c.epart + c.off_rbl;
  pa.nbr = nullptr;
  a.id = c.id[b];
  const double rc2 = c.rc * c.rc, rk2 = c.r_core * c.r_core;
  a.rcore2d = rk2; a.rs2d = rc2;
  a.p = c.p_rbl;
  a.key = make_uint2((uint32_t)c.seed, (uint32_t)(c.seed >> 32) ^ c.replica);
  a.step = c.step_dev;
  a.fsum_part = c.rbl_part;
  a.err = c.err;
  a.ncore = want_debug ? c.nbr : nullptr;
  a.nshell = want_debug ? c.nshell : nullptr;
  a.partners = want_debug ? c.partners : nullptr;
  const int64_t blocks = rbl_blocks(c.N);
  const bool multi = c.nt > 1, coul = c.Nq > 0;
  int gs;
  bool wrap;
  rbl_shape(c, &gs, &wrap);
  {
    // The classification compares an r^2 from FP32 frame coordinates with the bands: a
    // group's candidates lie within gs + 1 cells of its leader in x and 2 in y and z (L/2
    // in a wrapping box), and each band is at least that r^2's error bound.
    double X[3];
    for (int d = 0; d < 3; ++d) {
      const double w = c.box[d] / c.grid.n[d];
      X[d] = wrap ? 0.5 * c.box[d] : std::min((d == 0 ? gs + 1 : 2) * w, 0.5 * c.box[d]);
    }
    const double bk = frame_band(X, c.r_core, c.box, wrap), bs = frame_band(X, c.rc, c.box, wrap);
    a.rcore2_lo = (float)(rk2 * (1.0 - bk)); a.rcore2_hi = (float)(rk2 * (1.0 + bk));
    a.rs2_lo = (float)(rc2 * (1.0 - bs)); a.rs2_hi = (float)(rc2 * (1.0 + bs));
  }
  for (int d = 0; d < 3; ++d) {
    pa.L[d] = (float)c.box[d];
    pa.invL[d] = (float)(1.0 / c.box[d]);
  }
  a.gs = gs;
  a.masks = c.rbl_masks;
  a.slots = c.rbl_slots;
  a.nslots = (int)c.rbl_nslots;
  pa.smax = 1;
  pa.comp = c.precision == RBE_FP32_COMP;
  if (c.precision == RBE_FP64) rbl_launch<double>(a, blocks, coul, c.rbl_eager, multi, wrap, c.stream);
  else rbl_launch<float>(a, blocks, coul, c.rbl_eager, multi, wrap, c.stream);
  mark(c, RBE_PH_PAIR2);
  const int64_t ncomp = rbl_compact_count(blocks);
  rbl_compact_kernel<<<(unsigned)ncomp, 256, 0, c.stream>>>(c.epart + c.off_rbl, c.rbl_part, blocks,
                                                             (blocks + ncomp - 1) / ncomp,
                                                             c.rbl_cpart, c.rbl_cpart + ncomp * NQ_PAIR);
  rbl_mean_kernel<<<1, 256, 0, c.stream>>>(c.rbl_cpart + ncomp * NQ_PAIR, ncomp, c.N, c.rbl_mean);
  const unsigned nb = (unsigned)((c.N + 255) / 256);
  if (c.precision == RBE_FP64) rbl_subtract_kernel<double><<<nb, 256, 0, c.stream>>>(c.Fd, c.N, c.rbl_mean);
  else rbl_subtract_kernel<float><<<nb, 256, 0, c.stream>>>(c.F, c.N, c.rbl_mean);
  return cudaGetLastError();
}

}  // namespace rbe
