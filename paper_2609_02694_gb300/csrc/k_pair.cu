// k_pair.cu -- real-space pair forces over linked cells (Eqs. F_i, G_short, LJ).
//
// F_i += sum_{j != i, r_ij <= r_c} (C q_i q_j G(r) + G_LJ(r)) (r_i - r_j)
//   G(r)    = erfc(sqrt(alpha) r) / r^3 + 2 sqrt(alpha) exp(-alpha r^2) / (sqrt(pi) r^2)
//   G_LJ(r) = 24 eps (2 sigma^12 / r^14 - sigma^6 / r^8)
// with r_i - r_j the minimum image: on the 2^-32 grid that is the two's-complement
// difference of the fractional coordinates, so no image shifts are needed.
//
// Work decomposition (one thread per particle i, 32 consecutive cell-sorted particles per
// warp). Lanes sharing a cell row (c_y, c_z) form a group, and the group walks the union
// of its members' stencils: for every (dy, dz) row, one contiguous run of cells in x.
//  1. Stage: the warp loads 32 candidates j at a time (a chunk) into a ring of four
//     chunk positions in shared memory. Each lane converts one of them to coordinates
//     relative to the group leader: half-precision test copies, exact integers.
//  2. Test: every lane tests its own i against the staged j (broadcast reads, two
//     candidates per half-precision instruction) with a cutoff widened beyond the worst
//     rounding and collects a 32-bit hit mask, which it queues (one entry per chunk with
//     hits) in shared memory. Slots past the run and lanes outside the group get test
//     coordinates that can never hit.
//  3. Evaluate: before a chunk overwrites a ring position, the warp runs just enough
//     iterations that every lane has consumed its hits staged there; every lane with hits
//     pending evaluates in each iteration, so lanes light on old chunks work ahead. Each
//     lane recomputes the displacement exactly from the integer coordinates and applies
//     the exact cutoff decision: FP32 outside a band of at least +-1e-5 (its top is the
//     pre-test's threshold), FP64 inside it, which matches the oracle's decision bit for
//     bit. Then it evaluates the pair force.
// Forces are summed per i in a fixed j order with no atomics, so results are run-to-run
// reproducible. The hot loop is FP32 ALU / SFU bound.
// The BUILD variant walks the same windows with the list radius r_c + skin and, instead of
// evaluating, appends each hit j (in the same candidate order) to i's Verlet list.
#include <algorithm>
#include <climits>
#include <cmath>

#include "pair_common.cuh"

namespace rbe {

constexpr int kMaxRows = 49;            // (2R+1)^2 stencil rows for R <= 3
constexpr int kMaxSeg = 2 * kMaxRows;   // a row wraps into at most two runs of cells
constexpr int kWin = 4;                 // chunks of 32 candidates staged per window
constexpr int kHitQ = 4;                // hit-mask queue entries per lane (at most 4 pending)

// 28 warps per SM (at most 72 registers): occupancy is worth more than registers to this
// issue-bound loop (32 warps spill and run slower). One-warp blocks: a warp that finishes
// early frees its slot instead of waiting at a block barrier for the slowest warp.
template <typename real, bool LJ, bool COUL, bool MULTI, bool WRAP, bool T16, bool BUILD>
__device__ __forceinline__ void pair_body(const PairArgs &a, int bx, int) {
  __shared__ float4 stage[kPairWarps][kWin][T16 ? 1 : 32];     // FP32 test coordinates
  __shared__ uint4 stage16[kPairWarps][kWin][T16 ? 16 : 1];    // packed half test coordinates
  __shared__ int4 stage_d[kPairWarps][kWin][32];               // exact integer frame coords, type
  __shared__ float stage_q[kPairWarps][kWin][32];
  // candidate indices: read by the FP64 charge gather and by the list build only
  constexpr bool NEEDJ = BUILD || (COUL && sizeof(real) == 8);
  __shared__ int32_t stage_j[kPairWarps][kWin][NEEDJ ? 32 : 1];
  __shared__ int32_t seg_beg[kPairWarps][kMaxSeg];
  __shared__ int32_t seg_pre[kPairWarps][kMaxSeg + 1];
  __shared__ double wred[kPairWarps][NQ_PAIR];
  // per-lane queues of pending hit masks: entry e of lane l holds (mask, ring slot base) of
  // one chunk with hits; entry-major, so any mix of entries costs the minimum two wavefronts
  constexpr bool HL = !BUILD && !WRAP;
  __shared__ uint2 hitq[kPairWarps][HL ? kHitQ : 1][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const int64_t n = a.set.n;
  const int64_t i0 = ((int64_t)bx * kPairWarps + wid) * 32;
  const int64_t i = i0 + lane;
  const bool valid = i < n;
  const LJTable *tab = a.table;
  if (BUILD && *a.gate == 0) return;  // no list build this step (uniform over the grid)
  PairAcc<real> acc;
  acc.fx = acc.fy = acc.fz = acc.ulj = acc.wlj = acc.uc = acc.wc = (real)0;
  acc.cuc = acc.cwc = (real)0;
  acc.nbr = 0;
  int cnt = 0;  // BUILD: list length of i
  int32_t *lst = BUILD ? a.list + (i0 >> 5) * (int64_t)a.K * 32 + lane : nullptr;
  if (i0 < n) {
    const int n0 = a.grid.n[0], n1 = a.grid.n[1], n2 = a.grid.n[2];
    const int R0 = a.grid.R[0], R1 = a.grid.R[1], R2 = a.grid.R[2];
    const uint32_t sxi = valid ? a.set.sx[i] : 0u;
    const uint32_t syi = valid ? a.set.sy[i] : 0u;
    const uint32_t szi = valid ? a.set.sz[i] : 0u;
    real qi = (real)0;
    if (COUL && valid) qi = sizeof(real) == 8 ? (real)a.set.qd[i] : (real)a.set.qf[i];
    const int ti = (MULTI && valid) ? a.set.type[i] : 0;
    const int cx = cell_of(sxi, n0), cy = cell_of(syi, n1), cz = cell_of(szi, n2);
    const float rc2_hi = a.pc.rc2_hi;
    const int ny = 2 * R1 + 1, nrows = ny * (2 * R2 + 1);
    unsigned remaining = __ballot_sync(FULL, valid);
    while (remaining) {
      const int leader = __ffs(remaining) - 1;
      const int gy = __shfl_sync(FULL, cy, leader), gz = __shfl_sync(FULL, cz, leader);
      const int gx0 = __shfl_sync(FULL, cx, leader);
      const bool in = valid && cy == gy && cz == gz &&
                      (WRAP || cx - gx0 < (T16 ? a.smax16 : a.smax)) &&
                      ((remaining >> lane) & 1u);
      const unsigned gmask = __ballot_sync(FULL, in);
      remaining &= ~gmask;
      const int cxlo = __reduce_min_sync(FULL, in ? cx : INT_MAX);
      const int cxhi = __reduce_max_sync(FULL, in ? cx : INT_MIN);
      const uint32_t ox = __shfl_sync(FULL, sxi, leader);
      const uint32_t oy = __shfl_sync(FULL, syi, leader);
      const uint32_t oz = __shfl_sync(FULL, szi, leader);
      // integer frame coordinates relative to the leader (exact); float / half test copies
      const int dxi = (int)(sxi - ox), dyi = (int)(syi - oy), dzi = (int)(szi - oz);
      // test coordinates; lanes outside the group get a point that no candidate can reach
      const float far_i = T16 ? -30000.f : -1e30f;
      const float xi = (HL && !in) ? far_i : (float)dxi * a.pc.h[0];
      const float yi = (HL && !in) ? far_i : (float)dyi * a.pc.h[1];
      const float zi = (HL && !in) ? far_i : (float)dzi * a.pc.h[2];
      const __half2 xi2 = __float2half2_rn((HL && !in) ? far_i : xi * a.scale16);
      const __half2 yi2 = __float2half2_rn((HL && !in) ? far_i : yi * a.scale16);
      const __half2 zi2 = __float2half2_rn((HL && !in) ? far_i : zi * a.scale16);
      const __half2 thr2 = __float2half2_rn(66.5f);
      const int span = cxhi - cxlo + 2 * R0 + 1;
      // Trimming: every row of cells is sorted by x, so a row's run is cut to the x-range
      // that some member of the group can reach: members span [gxlo, gxhi] in x (frame
      // units), and a row whose cells lie at y/z distance d from the group's box reaches
      // only sqrt(r^2 - d^2) in x. (Not for the wrapping variant or a run that is a whole
      // row, whose frame coordinates are not monotone along the run.)
      const bool trim = !WRAP && a.trim && span < n0;
      const int gxlo = __reduce_min_sync(FULL, in ? dxi : INT_MAX);
      const int gxhi = __reduce_max_sync(FULL, in ? dxi : INT_MIN);
      const int gylo = __reduce_min_sync(FULL, in ? dyi : INT_MAX);
      const int gyhi = __reduce_max_sync(FULL, in ? dyi : INT_MIN);
      const int gzlo = __reduce_min_sync(FULL, in ? dzi : INT_MAX);
      const int gzhi = __reduce_max_sync(FULL, in ? dzi : INT_MIN);
      // 1. Runs of candidates: one lane per stencil row (dz, dy) loads the row's cell
      //    range(s) in parallel; a warp scan turns the run lengths into offsets.
      int carry = 0;
      for (int rb = 0; rb < nrows; rb += 32) {
        const int r = rb + lane;
        int b0 = 0, l0 = 0, b1 = 0, l1 = 0;
        if (r < nrows) {
          const int dz = r / ny - R2, dy = r % ny - R1;
          const int rz = ((gz + dz) % n2 + n2) % n2;
          const int ry = ((gy + dy) % n1 + n1) % n1;
          const int64_t rowbase = (int64_t)n0 * (ry + (int64_t)n1 * rz);
          int sa0, sb0, sa1 = 0, sb1 = -1;
          int64_t sh0 = 0, sh1 = 0;  // unwrapping shift of each segment (x past 0 or L)
          if (span >= n0) { sa0 = 0; sb0 = n0 - 1; }
          else {
            const int lo = cxlo - R0, hi = cxhi + R0;
            if (lo < 0) { sa0 = lo + n0; sb0 = n0 - 1; sa1 = 0; sb1 = hi; sh0 = -((int64_t)1 << 32); }
            else if (hi >= n0) { sa0 = lo; sb0 = n0 - 1; sa1 = 0; sb1 = hi - n0; sh1 = (int64_t)1 << 32; }
            else { sa0 = lo; sb0 = hi; }
          }
          b0 = a.set.cell_start[rowbase + sa0];
          l0 = a.set.cell_start[rowbase + sb0 + 1] - b0;
          if (sb1 >= sa1) {
            b1 = a.set.cell_start[rowbase + sa1];
            l1 = a.set.cell_start[rowbase + sb1 + 1] - b1;
          }
          if (trim) {
            // the row's y and z extent in frame units (cells gy + dy, gz + dz unwrapped;
            // edges rounded outward by 2 units), its distance from the group's box, and
            // the x-reach left (radius widened by 1e-9, reach rounded up, +2 units)
            const double wy = 4294967296.0 / n1, wz = 4294967296.0 / n2;
            const double ylo = (gy + dy) * wy - (double)oy - 2.0, yhi = (gy + dy + 1) * wy - (double)oy + 2.0;
            const double zlo = (gz + dz) * wz - (double)oz - 2.0, zhi = (gz + dz + 1) * wz - (double)oz + 2.0;
            const double ddy = fmax(0.0, fmax(ylo - gyhi, gylo - yhi)) * a.pc.hd[1];
            const double ddz = fmax(0.0, fmax(zlo - gzhi, gzlo - zhi)) * a.pc.hd[2];
            const double rx2 = a.pc.rc2d * (1.0 + 1e-9) - ddy * ddy - ddz * ddz;
            if (rx2 <= 0.0) {
              l0 = l1 = 0;
            } else {
              const double rx = ceil(sqrt(rx2) / a.pc.hd[0]) + 2.0;
              const int64_t xlo = (int64_t)gxlo - (int64_t)rx, xhi = (int64_t)gxhi + (int64_t)rx;
              // first member of [b, b + l) at unwrapped x (s_x + shift - o_x, exact) >= key.
              // Runs are sorted by s_x; the minimum-image frame coordinate is not monotone
              // along a run (candidates beyond L/2 of the leader wrap), the unwrapped one is.
              auto first_ge = [&](int b, int l, int64_t key, int64_t sh) {
                int lo = 0, hi = l;
                while (lo < hi) {
                  const int mid = (lo + hi) >> 1;
                  if ((int64_t)a.set.sx[b + mid] + sh - (int64_t)ox < key) lo = mid + 1;
                  else hi = mid;
                }
                return lo;
              };
              int u0 = first_ge(b0, l0, xlo, sh0), v0 = first_ge(b0, l0, xhi + 1, sh0);
              b0 += u0; l0 = v0 - u0;
              if (l1 > 0) {
                const int u1 = first_ge(b1, l1, xlo, sh1), v1 = first_ge(b1, l1, xhi + 1, sh1);
                b1 += u1; l1 = v1 - u1;
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
        if (r < nrows) {
          seg_beg[wid][2 * r] = b0;
          seg_pre[wid][2 * r] = excl;
          seg_beg[wid][2 * r + 1] = b1;
          seg_pre[wid][2 * r + 1] = excl + l0;
        }
        carry += __shfl_sync(FULL, incl, 31);
      }
      if (lane == 0) seg_pre[wid][2 * nrows] = carry;
      __syncwarp();
      const int T = carry;
      // Stage candidate c of the run (one per lane) at chunk position w of the ring, in two
      // parts so that the global loads of the next chunk can be in flight while this one is
      // tested: load (run search, coordinates, type, charge, index) and store (test
      // coordinates, exact integer frame coordinates and type, charge, index). Past the
      // run: a valid dummy (set index 0, type 0, no charge) with test coordinates that no
      // lane can reach. Idle lanes of the evaluation loops read some staged slot and gather
      // its charge or LJ-table entry by index before the result is masked, so no slot may
      // keep an index left by an earlier chunk or kernel.
      struct Cand { uint32_t x, y, z; int t; float q; int32_t j; bool v; };
      auto load_one = [&](int c, int &s, Cand &r) {
        r.v = c < T;
        r.x = r.y = r.z = 0u; r.t = 0; r.q = 0.f; r.j = 0;
        if (r.v) {
          while (seg_pre[wid][s + 1] <= c) ++s;
          const int64_t j = seg_beg[wid][s] + (c - seg_pre[wid][s]);
          r.x = a.set.sx[j]; r.y = a.set.sy[j]; r.z = a.set.sz[j];
          if (MULTI) r.t = a.set.type[j];
          if (COUL) r.q = a.set.qf[j];
          r.j = (int32_t)j;
        }
      };
      auto store_one = [&](int w, const Cand &r) {
        if (r.v) {
          const int dxj = (int)(r.x - ox), dyj = (int)(r.y - oy), dzj = (int)(r.z - oz);
          const float fx = (float)dxj * a.pc.h[0];
          const float fy = (float)dyj * a.pc.h[1];
          const float fz = (float)dzj * a.pc.h[2];
          if (T16) {
            // entry p packs candidates p (low halves) and p + 16 (high halves), so that
            // bit b of the test mask is candidate b
            __half *h = reinterpret_cast<__half *>(&stage16[wid][w][lane & 15]);
            const int o = lane >> 4;
            h[o] = __float2half_rn(fx * a.scale16);
            h[2 + o] = __float2half_rn(fy * a.scale16);
            h[4 + o] = __float2half_rn(fz * a.scale16);
          } else {
            stage[wid][w][lane] = make_float4(fx, fy, fz, 0.f);
          }
          stage_d[wid][w][lane] = make_int4(dxj, dyj, dzj, r.t);
        } else {
          if (T16) {
            __half *h = reinterpret_cast<__half *>(&stage16[wid][w][lane & 15]);
            const int o = lane >> 4;
            h[o] = h[2 + o] = h[4 + o] = __float2half_rn(30000.f);
          } else {
            stage[wid][w][lane] = make_float4(1e30f, 1e30f, 1e30f, 0.f);
          }
          stage_d[wid][w][lane] = make_int4(0, 0, 0, 0);
        }
        if (COUL) stage_q[wid][w][lane] = r.q;
        if (NEEDJ) stage_j[wid][w][lane] = r.j;
      };
      const int4 *sd = &stage_d[wid][0][0];
      const float *sq = &stage_q[wid][0][0];
      const int32_t *sj = &stage_j[wid][0][0];
      if (HL) {
        // 2. Chunks of 32 candidates through a ring of kWin staged chunks. Each lane tests
        //    every staged candidate, collects a 32-bit hit mask per chunk and queues it (with
        //    the chunk's ring position) when it is not empty. Before a chunk overwrites a ring
        //    position, the warp evaluates just enough iterations that every lane has consumed
        //    its hits staged there; each iteration takes the highest set bit of the lane's
        //    current mask, or the next queued mask when the current one is spent. Every lane
        //    with anything pending evaluates in each iteration, so a lane that is light on the
        //    oldest chunk works ahead on newer ones: the warp's trip count follows its
        //    heaviest lane over four chunks. Each lane evaluates its hits in a fixed order
        //    (chunks in order, within a chunk the highest candidate first).
        //    At most four masks are queued: after a drain only the three newest chunks can
        //    hold pending hits, and the chunk being tested adds one.
        int hd = 0, tl = 0, cnt = 0;  // queue read and write count, pending hits
        uint32_t cm = 0u;             // the mask being consumed (0: take the next queued one)
        int cp = 0;                   // its ring slot base (ring position * 32)
        uint32_t q4 = 0u;             // hits per ring position (8-bit fields)
        const int nch = (T + 31) >> 5;
        int sg = 0;
        Cand nx;  // the next chunk's candidate of this lane, loaded ahead
        {
          int s = sg;
          load_one(lane, s, nx);
          sg = __shfl_sync(FULL, s, 31);
        }
        for (int ch = 0; ch <= nch; ++ch) {
          const int p = ch & (kWin - 1);
          if (ch >= kWin || ch == nch) {
            // The pending hits of ring position p (chunk ch - kWin) are the oldest ones:
            // all pending minus those of the newer chunks. After the last chunk: all.
            int need = cnt;
            if (ch < nch) {
              const int newer = (int)((q4 * 0x01010101u) >> 24) - (int)((q4 >> (8 * p)) & 0xffu);
              need = max(0, cnt - newer);
            }
            const int nit = __reduce_max_sync(FULL, need);
            const int dummy = ((ch - 1) & (kWin - 1)) * 32;  // a slot of the latest chunk
            for (int k = 0; k < nit; ++k) {
              const bool act = k < cnt;
              const uint2 e = hitq[wid][hd & (kHitQ - 1)][lane];
              const bool take = act && cm == 0u;
              cm = take ? e.x : cm;
              cp = take ? (int)e.y : cp;
              hd += take ? 1 : 0;
              const int hb = 31 - __clz(cm);  // highest pending candidate first (one FLO)
              const int slot = act ? cp + hb : dummy;
              cm &= ~(1u << (hb & 31));
              const int4 d = sd[slot];
              const int dsx = (int)((uint32_t)dxi - (uint32_t)d.x);
              const int dsy = (int)((uint32_t)dyi - (uint32_t)d.y);
              const int dsz = (int)((uint32_t)dzi - (uint32_t)d.z);
              real qj = (real)0;
              if (COUL) qj = sizeof(real) == 8 ? (real)a.set.qd[sj[slot]] : (real)sq[slot];
              // (the particle itself, at zero displacement, is excluded by the evaluation)
              pair_eval_masked<real, LJ, COUL, MULTI>(a, tab, act, dsx, dsy, dsz, qi, ti, qj,
                                                      d.w, acc);
            }
            cnt = max(0, cnt - nit);
            __syncwarp();  // position p is free for every lane
          }
          if (ch == nch) break;
          store_one(p, nx);
          if (ch + 1 < nch) {
            int s = sg;
            load_one(32 * (ch + 1) + lane, s, nx);
            sg = __shfl_sync(FULL, s, 31);
          }
          __syncwarp();
          // test: bit b of mk is candidate b of the chunk
          uint32_t mk = 0u;
          if (T16) {
#pragma unroll
            for (int pp = 0; pp < 16; ++pp) {
              const uint4 v = stage16[wid][p][pp];
              const __half2 dx2 = __hsub2(xi2, *reinterpret_cast<const __half2 *>(&v.x));
              const __half2 dy2 = __hsub2(yi2, *reinterpret_cast<const __half2 *>(&v.y));
              const __half2 dz2 = __hsub2(zi2, *reinterpret_cast<const __half2 *>(&v.z));
              const __half2 r2 = __hfma2(dx2, dx2, __hfma2(dy2, dy2, __hmul2(dz2, dz2)));
              mk |= __hlt2_mask(r2, thr2) & (0x00010001u << pp);  // one LOP3 (pp unrolled)
            }
          } else {
#pragma unroll
            for (int tt = 0; tt < 32; ++tt) {
              const float4 q = stage[wid][p][tt];
              const float ddx = xi - q.x, ddy = yi - q.y, ddz = zi - q.z;
              const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
              mk |= r2 < rc2_hi ? (1u << tt) : 0u;
            }
          }
          if (mk != 0u) {
            hitq[wid][tl & (kHitQ - 1)][lane] = make_uint2(mk, (uint32_t)(p * 32));
            ++tl;
          }
          const int nh = __popc(mk);
          cnt += nh;
          q4 = (q4 & ~(0xffu << (8 * p))) | ((uint32_t)nh << (8 * p));
        }
        continue;
      }
      // 2. (Lists and small boxes.) Windows of kWin chunks of 32 candidates: stage, test
      //    every staged candidate against the lane's own i (bit masks), then evaluate (or
      //    list) the hits directly from the staged exact coordinates.
      int sg = 0;
      for (int base = 0; base < T; base += 32 * kWin) {
#pragma unroll
        for (int w = 0; w < kWin; ++w) {
          int s = sg;
          Cand r;
          load_one(base + 32 * w + lane, s, r);
          sg = __shfl_sync(FULL, s, 31);
          store_one(w, r);
        }
        __syncwarp();
        uint32_t m[kWin];
#pragma unroll
        for (int w = 0; w < kWin; ++w) {
          const int nj = max(0, min(32, T - base - 32 * w));
          uint32_t mask = 0u;
          if (nj > 0) {
            if (T16) {
              // bit p: candidate p, bit 16 + p: candidate p + 16
#pragma unroll
              for (int pp = 0; pp < 16; ++pp) {
                const uint4 v = stage16[wid][w][pp];
                const __half2 dx2 = __hsub2(xi2, *reinterpret_cast<const __half2 *>(&v.x));
                const __half2 dy2 = __hsub2(yi2, *reinterpret_cast<const __half2 *>(&v.y));
                const __half2 dz2 = __hsub2(zi2, *reinterpret_cast<const __half2 *>(&v.z));
                const __half2 r2 = __hfma2(dx2, dx2, __hfma2(dy2, dy2, __hmul2(dz2, dz2)));
                mask |= __hlt2_mask(r2, thr2) & (0x00010001u << pp);  // one LOP3 (pp unrolled)
              }
              if (nj < 32) mask &= (1u << nj) - 1u;
            } else {
#pragma unroll
              for (int tt = 0; tt < 32; ++tt) {
                const float4 p = stage[wid][w][tt];
                float ddx = xi - p.x, ddy = yi - p.y, ddz = zi - p.z;
                if (WRAP) {
                  ddx = fold(ddx, a.L[0], a.invL[0]);
                  ddy = fold(ddy, a.L[1], a.invL[1]);
                  ddz = fold(ddz, a.L[2], a.invL[2]);
                }
                const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
                mask |= (r2 < rc2_hi) ? (1u << tt) : 0u;
              }
              if (nj < 32) mask &= (1u << nj) - 1u;
            }
          }
          m[w] = in ? mask : 0u;
        }
        // evaluate the hits of the window (each lane its own, in candidate order); idle
        // lanes run a masked dummy so the loop body has no divergent branch
        uint64_t mA = (uint64_t)m[0] | ((uint64_t)m[1] << 32);
        uint64_t mB = (uint64_t)m[2] | ((uint64_t)m[3] << 32);
        // uniform trip count: the largest number of hits of any lane in this window
        const int nhit = __reduce_max_sync(FULL, __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]));
        for (int k = 0; k < nhit; ++k) {
          const bool useA = mA != 0ull;
          const uint64_t bits = useA ? mA : mB;
          const bool act = bits != 0ull;
          const int b = act ? __ffsll((long long)bits) - 1 : 0;
          const uint64_t rest = bits & (bits - 1ull);
          mA = useA ? rest : mA;
          mB = useA ? mB : rest;
          const int slot = (useA ? 0 : 64) + b;  // window slot = chunk * 32 + candidate
          const int4 d = sd[slot];
          const int dsx = (int)((uint32_t)dxi - (uint32_t)d.x);
          const int dsy = (int)((uint32_t)dyi - (uint32_t)d.y);
          const int dsz = (int)((uint32_t)dzi - (uint32_t)d.z);
          if (BUILD) {
            const int32_t j = sj[slot];
            const float ex = (float)dsx * a.pc.h[0];
            const float ey = (float)dsy * a.pc.h[1];
            const float ez = (float)dsz * a.pc.h[2];
            const bool hit = act && j != (int32_t)i && mad(ex, ex, mad(ey, ey, ez * ez)) <= a.pc.rc2_hi;
            if (hit && cnt < a.K) lst[(int64_t)cnt * 32] = j;
            cnt += hit ? 1 : 0;
          } else {
            real qj = (real)0;
            if (COUL) qj = sizeof(real) == 8 ? (real)a.set.qd[sj[slot]] : (real)sq[slot];
            // the particle itself, at zero displacement, is excluded by the evaluation
            // (coincident particles, which no valid configuration has, would be too)
            pair_eval_masked<real, LJ, COUL, MULTI>(a, tab, act, dsx, dsy, dsz, qi, ti, qj, d.w,
                                                    acc);
          }
        }
        __syncwarp();
      }
    }
    if (BUILD) {
      if (valid) a.len[i] = min(cnt, a.K);
      const int mx = __reduce_max_sync(FULL, valid ? cnt : 0);
      if (lane == 0) {
        atomicMax(a.maxlen, mx);
        if (mx > a.K) atomicOr(a.err, ERRBIT_CAPACITY);
      }
    } else if (valid) {
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
  }
  if (BUILD) return;
  // block partials of the energies and virials (halves of the per-i sums)
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
    a.epart[(int64_t)bx * NQ_PAIR + threadIdx.x] = 0.5 * s;
  }
}

template <typename real, bool LJ, bool COUL, bool MULTI, bool WRAP, bool T16, bool BUILD>
__global__ void __launch_bounds__(kPairWarps * 32, 28 / kPairWarps) pair_kernel(const PairArgs a) {
  pair_body<real, LJ, COUL, MULTI, WRAP, T16, BUILD>(a, (int)blockIdx.x, (int)gridDim.x);
}

template <typename real, bool LJ, bool COUL, bool BUILD = false>
static cudaError_t launch_one(Ctx &c, const PairArgs &a, int64_t n, bool multi, bool wrap) {
  const unsigned blocks = (unsigned)((n + 32 * kPairWarps - 1) / (32 * kPairWarps));
  if (blocks == 0) return cudaSuccess;
  const dim3 g(blocks), b(kPairWarps * 32);
  // (per replica in a batch; the list build is not used batched)
#define RBE_PK(MU, WR, T)                                                                     \
  dispatch(c, pair_kernel<real, LJ, COUL, MU, WR, T, BUILD>,                                  \
           nullptr, g, b, 0, a, !BUILD)
  if (wrap) return multi ? RBE_PK(true, true, false) : RBE_PK(false, true, false);
  if (a.smax16 > 0) return multi ? RBE_PK(true, false, true) : RBE_PK(false, false, true);
  return multi ? RBE_PK(true, false, false) : RBE_PK(false, false, false);
#undef RBE_PK
}

// Group x-extent (cells) for the half-precision test at cutoff rc with stencil R: every
// frame coordinate of a group and its candidates stays below 64 scaled units (rc = 8),
// i.e. 8 rc in length; 0 disables the half test (the FP32 test is used).
int frame_span_cells_half(const Ctx &c, int smax, double rc, const int *R) {
  if (smax < 1) return 0;
  const double lim = 8.0 * rc * (1.0 - 1e-6);
  for (int d = 1; d < 3; ++d)
    if ((2 * R[d] + 2) * (c.box[d] / c.grid.n[d]) >= lim) return 0;
  const double ax = c.box[0] / c.grid.n[0];
  const int s = (int)std::floor(lim / ax) - 2 * R[0] - 1;
  return s >= 1 ? std::min(s, smax) : 0;
}

// Largest x-extent (in cells) of a group whose leader frame stays a valid minimum image at
// cutoff rc; 0 when even one cell is too wide (the wrapping variant is used then).
int frame_span_cells(const Ctx &c, double rc) {
  for (int d = 1; d < 3; ++d) {
    const double a = c.box[d] / c.grid.n[d];
    if (!(a + rc < 0.5 * c.box[d] * (1.0 - 1e-9))) return 0;
  }
  const double ax = c.box[0] / c.grid.n[0];
  const int s = (int)std::floor((0.5 * c.box[0] * (1.0 - 1e-9) - rc) / ax);
  return s >= 1 ? std::min(s, 1 << 20) : 0;
}

int64_t pair_blocks(int64_t n) { return (n + 32 * kPairWarps - 1) / (32 * kPairWarps); }

// An FP32 r^2 formed from FP32 frame coordinates (each the integer offset from the group
// leader, converted and scaled by L / 2^32: within 2u|x| of exact, u = 2^-24) is off by at
// most, per axis, e_d = 4u X_d (both ends) + 2u r (the rounded difference and the rounded
// scale), plus u L_d when the difference is folded into the box; so the sum of squares is
// within 2 r |e| + |e|^2, and the fused sums add 3u r^2 more. The band is that bound, taken
// 1.25 times and never below 1e-5, relative to r^2: outside it the FP32 comparison is exact.
double frame_band(const double X[3], double r, const double box[3], bool wrap) {
  const double u = std::ldexp(1.0, -24);
  double s2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double e = 4.0 * u * X[d] + 2.0 * u * r + (wrap ? 2.0 * u * box[d] : 0.0);
    s2 += e * e;
  }
  const double eps = 2.0 * std::sqrt(s2) / r + s2 / (r * r) + 5.0 * u;
  return std::max(1e-5, 1.25 * eps);
}

// The FP32 pre-test compares an r^2 from FP32 frame coordinates with rc2_hi. A group's frame
// coordinates lie within (span + R) cells of its leader in x (span = smax16 for the half test,
// else smax) and R + 1 cells in y and z, or L/2 in a wrapping box, so rc2_hi is raised by the
// band for that extent. rc2_hi is also the top of the evaluation's exact band, which then
// only sends a few more pairs to the FP64 decision.
static void set_pretest_band(const Ctx &c, PairArgs &a, double r, bool wrap) {
  double X[3];
  const int span = a.smax16 > 0 ? a.smax16 : a.smax;
  for (int d = 0; d < 3; ++d) {
    const double w = c.box[d] / c.grid.n[d];
    const int cells = d == 0 ? span + a.grid.R[0] : a.grid.R[d] + 1;
    X[d] = wrap ? 0.5 * c.box[d] : std::min(cells * w, 0.5 * c.box[d]);
  }
  a.pc.rc2_hi = (float)(r * r * (1.0 + frame_band(X, r, c.box, wrap)));
}

cudaError_t launch_pair(Ctx &c, bool want_counts) {
  const int b = c.cur;
  const bool fused = c.Nq * 2 > c.N;  // most particles charged: one LJ + Coulomb pass
  const bool multi = c.nt > 1;
  PairArgs a;
  a.grid = c.grid;
  a.pc = c.pc;
  a.ljA = c.lj.A[0]; a.ljB = c.lj.B[0]; a.ljA12 = c.lj.A12[0]; a.ljB6 = c.lj.B6[0];
  a.ljAd = c.lj.Ad[0]; a.ljBd = c.lj.Bd[0]; a.ljA12d = c.lj.A12d[0]; a.ljB6d = c.lj.B6d[0];
  a.table = reinterpret_cast<const LJTable *>(c.lj_dev);
  a.F = c.F; a.Fd = c.Fd; a.Fstride = c.N;
  // full set
  a.set.sx = c.s[b]; a.set.sy = c.s[b] + c.N; a.set.sz = c.s[b] + 2 * c.N;
  a.set.qf = c.qf[b]; a.set.qd = c.qd[b]; a.set.type = c.type[b];
  a.set.cell_start = c.cell_start; a.set.map = nullptr; a.set.n = c.N;
  a.accumulate = 0;
  a.epart = c.epart + c.off_pair;
  a.nbr = want_counts ? c.nbr : nullptr;
  a.smax = frame_span_cells(c, c.rc);
  a.comp = c.precision == RBE_FP32_COMP;
  a.scale16 = (float)(8.0 / c.rc);
  a.smax16 = c.pair_test16 ? frame_span_cells_half(c, a.smax, c.rc, c.grid.R) : 0;
  a.trim = 1;
  const bool wrap = a.smax == 0;
  for (int d = 0; d < 3; ++d) {
    a.L[d] = (float)c.box[d];
    a.invL[d] = (float)(1.0 / c.box[d]);
  }
  set_pretest_band(c, a, c.rc, wrap);
  const bool fp64 = c.precision == RBE_FP64;
  if (fused) {
    const cudaError_t e = fp64 ? launch_one<double, true, true>(c, a, c.N, multi, wrap)
                               : launch_one<float, true, true>(c, a, c.N, multi, wrap);
    if (e != cudaSuccess) return e;
  } else {
    const cudaError_t e = fp64 ? launch_one<double, true, false>(c, a, c.N, multi, wrap)
                               : launch_one<float, true, false>(c, a, c.N, multi, wrap);
    if (e != cudaSuccess) return e;
  }
  zero_partials_tail(c, c.off_pair, pair_blocks(c.N), c.n_pair_blk);
  mark(c, RBE_PH_PAIR2);
  // the charged subset's Coulomb pass (k_coul.cu), added to the forces the main pass wrote
  if (!fused && c.Nq > 0) return launch_coulomb_subset(c, c.cq4, false);
  return cudaGetLastError();
}

// The cluster kernel's pass (k_cpair.cu): each pair once, into the 64-bit fixed-point sums;
// then, when most particles carry no charge, the charged subset's Coulomb pass into the same
// sums. The k-space gather adds to them too, and launch_cluster_finish turns them into F.
cudaError_t launch_pair_cluster(Ctx &c, bool want_counts) {
  const bool fused = c.Nq * 2 > c.N;
  cudaError_t e = launch_cluster_pair(c, fused, c.nt > 1, want_counts);
  if (e != cudaSuccess) return e;
  mark(c, RBE_PH_PAIR2);
  if (!fused && c.Nq > 0) return launch_coulomb_subset(c, c.cq4, true);
  return cudaGetLastError();
}

// Verlet-list build at r_list = r_c + skin over the full set and, when the Coulomb pass
// runs separately, over the charged subset. Gated on the device rebuild flag.
cudaError_t launch_list_build(Ctx &c) {
  const int b = c.cur;
  const bool fused = c.Nq * 2 > c.N;
  PairArgs a{};
  a.grid = c.grid;
  for (int d = 0; d < 3; ++d) a.grid.R[d] = c.vl_R[d];
  a.pc = c.pc;
  const double rl = c.rc + c.vl_skin, rl2 = rl * rl;
  a.pc.rc2d = rl2;
  a.pc.rc2_lo = (float)(rl2 * (1.0 - 1e-5));  // (rc2_hi: the pre-test band, set below)
  a.set.sx = c.s[b]; a.set.sy = c.s[b] + c.N; a.set.sz = c.s[b] + 2 * c.N;
  a.set.qf = c.qf[b]; a.set.qd = c.qd[b]; a.set.type = nullptr;
  a.set.cell_start = c.cell_start; a.set.map = nullptr; a.set.n = c.N;
  a.smax = frame_span_cells(c, rl);
  a.scale16 = (float)(8.0 / rl);
  a.smax16 = c.pair_test16 ? frame_span_cells_half(c, a.smax, rl, c.vl_R) : 0;
  a.trim = 1;
  const bool wrap = a.smax == 0;
  for (int d = 0; d < 3; ++d) {
    a.L[d] = (float)c.box[d];
    a.invL[d] = (float)(1.0 / c.box[d]);
  }
  set_pretest_band(c, a, rl, wrap);
  a.list = c.vl_list; a.len = c.vl_len; a.K = c.vl_K;
  a.gate = c.vl_flags; a.maxlen = c.vl_flags + 2; a.err = c.err;
  cudaError_t e = launch_one<float, false, false, true>(c, a, c.N, false, wrap);
  if (e != cudaSuccess) return e;
  if (!fused && c.Nq > 0) {
    PairArgs q = a;
    q.set.sx = c.cs; q.set.sy = c.cs + c.Nq; q.set.sz = c.cs + 2 * c.Nq;
    q.set.qf = c.cqf; q.set.qd = c.cqd; q.set.type = nullptr;
    q.set.cell_start = c.ccell_start; q.set.map = c.cmap; q.set.n = c.Nq;
    q.list = c.vl_listq; q.len = c.vl_lenq; q.K = c.vl_Kq; q.maxlen = c.vl_flags + 3;
    e = launch_one<float, false, false, true>(c, q, c.Nq, false, wrap);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace rbe
