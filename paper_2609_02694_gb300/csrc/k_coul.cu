// k_coul.cu -- real-space Coulomb forces among the charged particles (Eqs. F_i, G_short):
//
//   F_i += sum_{j charged, j != i, r_ij <= r_c} C q_i q_j G(r) (r_i - r_j),
//   G(r) = erfc(sqrt(alpha) r) / r^3 + 2 sqrt(alpha / pi) exp(-alpha r^2) / r^2,
//
// the pass that follows the LJ pass when a minority of the particles carries charge. The
// charged subset is dilute (about one particle per cell of r_c / 2 at 10% charged), so a
// thread per particle would spend most of its time testing candidates its neighbours in the
// warp need and it does not. Here a warp serves one charged particle i:
//  1. Stencil: one lane per row (dy, dz) of cells finds the x-cells of the row within r_c of
//     i (a row farther than r_c is skipped), as at most two runs of the subset's
//     cell-ordered particles; a warp scan flattens the runs into one candidate list.
//  2. Test: 32 candidates at a time, one per lane, from their packed (s, q) records: the
//     exact minimum-image integer displacement, the cutoff decided in FP32 outside a band
//     around r_c^2 and by the oracle's FP64 expression inside it (always FP64 in the FP64
//     form). Hits are compacted (ballot) into a small per-warp buffer in shared memory.
//  3. Evaluate: whenever 32 hits are buffered (and once at the end) every lane evaluates one
//     of them (erfc, exp and a reciprocal square root), so the expensive terms run on full
//     warps. A warp sum gives F_i, added to the force of i's slot in the full set: to F after
//     a pass that wrote F, or to the cluster kernel's 64-bit fixed-point sums (three integer
//     atomics per particle, whose sums do not depend on their order).
// Each pair is evaluated from both sides, so the forces are reproducible run to run; the
// energy and virial partials take half of the per-i sums.
#include <climits>
#include <cmath>

#include "pair_common.cuh"

namespace rbe {

constexpr int kCoulWarps = 4;     // warps (charged particles) per block
constexpr int kCoulBuf = 64;      // buffered hits per warp (at most 31 pending + 32 new)
constexpr int kCoulMaxRows = 49;  // (2R+1)^2 stencil rows for R <= 3

struct CoulArgs {
  const uint4 *s4;            // charged subset, sorted: (s_x, s_y, s_z, q bits)
  const double *qd;           // FP64 charges of the subset (FP64 form)
  const int32_t *cell_start;  // the subset's cell starts (ncell + 1)
  const int32_t *map;         // subset slot -> slot of the full sorted set
  int64_t nq;
  Grid grid;
  PairConst pc;
  float *F;
  double *Fd;
  int64_t Fstride;
  double *epart;              // per-block partials (NQ_PAIR doubles)
  int comp;                   // Kahan-compensated energy and virial sums
  float reach2;               // r_c^2 widened: rows and cells farther than this are skipped
  long long *facc;            // nullable: 3 x N fixed-point force sums of the full set (then
  float fscale;               //   F is not written), their scale (FP32 forms)
  double fscale_d;            //   (FP64 form)
  int *err;                   //   (a sum out of range sets ERRBIT_NONFINITE)
};

int64_t coul_blocks(int64_t nq) { return (nq + kCoulWarps - 1) / kCoulWarps; }

template <typename real>
__device__ __forceinline__ void coul_body(const CoulArgs a, int bx, int) {
  constexpr bool F64 = sizeof(real) == 8;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ int4 buf[kCoulWarps][kCoulBuf];  // hits: integer displacement, charge bits or index
  __shared__ int32_t seg_beg[kCoulWarps][2 * kCoulMaxRows];
  __shared__ int32_t seg_pre[kCoulWarps][2 * kCoulMaxRows + 1];
  __shared__ double wred[kCoulWarps][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const PairConst &pc = a.pc;
  const int64_t i = (int64_t)bx * kCoulWarps + wid;
  real fx = (real)0, fy = (real)0, fz = (real)0;
  real uc = (real)0, wc = (real)0, cuc = (real)0, cwc = (real)0;
  if (i < a.nq) {
    const uint4 pi = a.s4[i];
    const real qi = F64 ? (real)a.qd[i] : (real)__uint_as_float(pi.w);
    const int n0 = a.grid.n[0], n1 = a.grid.n[1], n2 = a.grid.n[2];
    const int R1 = a.grid.R[1], R2 = a.grid.R[2];
    const int cy = cell_of(pi.y, n1), cz = cell_of(pi.z, n2);
    const int ny = 2 * R1 + 1, nrows = ny * (2 * R2 + 1);
    // t / ny as (t m) >> 8, m = ceil(256 / ny): exact for t < 64 and ny in {1, 3, 5, 7}
    const int mny = (256 + ny - 1) / ny;
    // i's y and z in cell units, and the cell widths
    const float fyc = (float)pi.y * ((float)n1 * 2.3283064365386963e-10f);
    const float fzc = (float)pi.z * ((float)n2 * 2.3283064365386963e-10f);
    const float wy = pc.h[1] * (4294967296.0f / (float)n1), wz = pc.h[2] * (4294967296.0f / (float)n2);
    int carry = 0;
    for (int rb = 0; rb < nrows; rb += 32) {
      const int t = rb + lane;
      int b0 = 0, l0 = 0, b1 = 0, l1 = 0;
      if (t < nrows) {
        const int tq = (t * mny) >> 8;
        const int dz = tq - R2, dy = t - tq * ny - R1;
        // distance of i from the row's cells in y and z, in cell widths (i's position in cell
        // units is within about 1e-5 cells in FP32; the distance is shrunk by 1e-3 cells)
        const float ey = fmaxf(0.f, fmaxf((float)(cy + dy) - fyc, fyc - (float)(cy + dy + 1)) - 1e-3f);
        const float ez = fmaxf(0.f, fmaxf((float)(cz + dz) - fzc, fzc - (float)(cz + dz + 1)) - 1e-3f);
        const float dyl = ey * wy, dzl = ez * wz;
        const float rx2 = mad(-dzl, dzl, mad(-dyl, dyl, a.reach2));
        if (rx2 > 0.f) {
          // periodic row indices (|dy| <= R1 < n1, |dz| <= R2 < n2)
          int ryw = cy + dy, rzw = cz + dz;
          ryw += ryw < 0 ? n1 : 0;
          ryw -= ryw >= n1 ? n1 : 0;
          rzw += rzw < 0 ? n2 : 0;
          rzw -= rzw >= n2 ? n2 : 0;
          const int64_t rowbase = (int64_t)n0 * (ryw + (int64_t)n1 * rzw);
          // x-cells within reach (unwrapped floor division by the cell width)
          const int64_t reach = (int64_t)(sqrtf(rx2) * (1.0f + 1e-5f) / pc.h[0]) + 4;
          const int64_t c0 = (((int64_t)pi.x - reach) * n0) >> 32;
          const int64_t c1 = (((int64_t)pi.x + reach) * n0) >> 32;
          int sa0, sb0, sa1 = 0, sb1 = -1;
          if (c1 - c0 + 1 >= n0) { sa0 = 0; sb0 = n0 - 1; }
          else if (c0 < 0) { sa0 = (int)(c0 + n0); sb0 = n0 - 1; sa1 = 0; sb1 = (int)c1; }
          else if (c1 >= n0) { sa0 = (int)c0; sb0 = n0 - 1; sa1 = 0; sb1 = (int)(c1 - n0); }
          else { sa0 = (int)c0; sb0 = (int)c1; }
          b0 = a.cell_start[rowbase + sa0];
          l0 = a.cell_start[rowbase + sb0 + 1] - b0;
          if (sb1 >= sa1) {
            b1 = a.cell_start[rowbase + sa1];
            l1 = a.cell_start[rowbase + sb1 + 1] - b1;
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
      if (t < nrows) {
        seg_beg[wid][2 * t] = b0;
        seg_pre[wid][2 * t] = excl;
        seg_beg[wid][2 * t + 1] = b1;
        seg_pre[wid][2 * t + 1] = excl + l0;
      }
      carry += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) seg_pre[wid][2 * nrows] = carry;
    __syncwarp();
    const int T = carry;
    // evaluate buffered hits [0, n) (one per lane)
    auto evaluate = [&](int n) {
      if (lane < n) {
        const int4 e = buf[wid][lane];
        real dx, dy, dz, r2, qj;
        if (F64) {
          dx = (real)__dmul_rn((double)e.x, pc.hd[0]);
          dy = (real)__dmul_rn((double)e.y, pc.hd[1]);
          dz = (real)__dmul_rn((double)e.z, pc.hd[2]);
          r2 = (real)__dadd_rn(__dadd_rn(__dmul_rn((double)dx, (double)dx),
                                         __dmul_rn((double)dy, (double)dy)),
                               __dmul_rn((double)dz, (double)dz));
          qj = (real)a.qd[e.w];
        } else {
          dx = (real)((float)e.x * pc.h[0]);
          dy = (real)((float)e.y * pc.h[1]);
          dz = (real)((float)e.z * pc.h[2]);
          r2 = mad(dx, dx, mad(dy, dy, dz * dz));
          qj = (real)__int_as_float(e.w);
        }
        real r, rinv, erfcv, expv;
        if (F64) {
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
        const real Cqq = (F64 ? (real)pc.C_d : (real)pc.C) * qi * qj;
        const real tsp = F64 ? (real)pc.two_sqrt_alpha_over_sqrt_pi_d
                             : (real)pc.two_sqrt_alpha_over_sqrt_pi;
        const real rinv2 = rinv * rinv;
        const real gc = Cqq * mad(erfcv * rinv, rinv2, tsp * expv * rinv2);
        fx = mad(gc, dx, fx); fy = mad(gc, dy, fy); fz = mad(gc, dz, fz);
        if (a.comp) {
          kahan_add(uc, cuc, Cqq * erfcv * rinv);
          kahan_add(wc, cwc, gc * r2);
        } else {
          uc = mad(Cqq * erfcv, rinv, uc);
          wc = mad(gc, r2, wc);
        }
      }
    };
    int nb = 0;  // buffered hits (warp-uniform)
    const int nseg = 2 * nrows;
    for (int base = 0; base < T; base += 32) {
      const int cc = base + lane;
      bool hit = false;
      int4 rec = make_int4(0, 0, 0, 0);
      if (cc < T) {
        // candidate cc's run: the last of the (possibly empty) runs starting at or before cc,
        // by a binary search over the run offsets (the same steps on every lane)
        int s = 0, hi = nseg;
        while (hi - s > 1) {
          const int mid = (s + hi) >> 1;
          if (seg_pre[wid][mid] <= cc) s = mid; else hi = mid;
        }
        const int64_t j = seg_beg[wid][s] + (cc - seg_pre[wid][s]);
        if (j != i) {
          const uint4 pj = a.s4[j];
          const int dsx = (int)(pi.x - pj.x), dsy = (int)(pi.y - pj.y), dsz = (int)(pi.z - pj.z);
          if (F64) {
            hit = exact_r2(pc, dsx, dsy, dsz) <= pc.rc2d;
          } else {
            const float ex = (float)dsx * pc.h[0], ey = (float)dsy * pc.h[1],
                        ez = (float)dsz * pc.h[2];
            const float r2 = mad(ex, ex, mad(ey, ey, ez * ez));
            hit = r2 < pc.rc2_lo;
            if (r2 >= pc.rc2_lo && r2 <= pc.rc2_hi) hit = exact_r2(pc, dsx, dsy, dsz) <= pc.rc2d;
          }
          rec = make_int4(dsx, dsy, dsz, F64 ? (int)j : (int)pj.w);
        }
      }
      const unsigned hm = __ballot_sync(FULL, hit);
      if (hit) buf[wid][nb + __popc(hm & ((1u << lane) - 1u))] = rec;
      nb += __popc(hm);
      __syncwarp();
      if (nb >= 32) {
        evaluate(32);
        const int4 keep = lane + 32 < nb ? buf[wid][lane + 32] : make_int4(0, 0, 0, 0);
        __syncwarp();
        if (lane + 32 < nb) buf[wid][lane] = keep;
        nb -= 32;
        __syncwarp();
      }
    }
    evaluate(nb);
    fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
    if (a.facc) {  // one component per lane (every lane holds the sums)
      if (lane < 3) {
        const real sc = F64 ? (real)a.fscale_d : (real)a.fscale;
        fx_add_i32(a.facc + lane * a.Fstride + a.map[i], lane == 0 ? fx : (lane == 1 ? fy : fz),
                   sc, a.err);
      }
    } else if (lane == 0) {
      const int64_t o = a.map[i];
      const int64_t S = a.Fstride;
      if (F64) {
        a.Fd[o] += (double)fx; a.Fd[S + o] += (double)fy; a.Fd[2 * S + o] += (double)fz;
      } else {
        a.F[o] += (float)fx; a.F[S + o] += (float)fy; a.F[2 * S + o] += (float)fz;
      }
    }
  }
  // block partials of the Coulomb energy and virial (halves of the per-i sums)
  const double u = warp_sum((double)uc - (double)cuc), w = warp_sum((double)wc - (double)cwc);
  if (lane == 0) { wred[wid][0] = u; wred[wid][1] = w; }
  __syncthreads();
  if (threadIdx.x < NQ_PAIR) {
    double s = 0.0;
    if (threadIdx.x == Q_UREAL || threadIdx.x == Q_WREAL)
      for (int k = 0; k < kCoulWarps; ++k) s += wred[k][threadIdx.x == Q_UREAL ? 0 : 1];
    a.epart[(int64_t)bx * NQ_PAIR + threadIdx.x] = 0.5 * s;
  }
}

// (16 blocks of 4 warps in the FP32 forms: the whole SM's 64 warps; the pass is bound by the
// latency of each warp's dependent loads, so occupancy is what hides it; 8 in the FP64 form,
// whose registers would spill)
template <typename real>
__global__ void __launch_bounds__(kCoulWarps * 32, sizeof(real) == 8 ? 8 : 16)
    coul_kernel(const CoulArgs a) {
  coul_body<real>(a, (int)blockIdx.x, (int)gridDim.x);
}


cudaError_t launch_coulomb_subset(Ctx &c, const uint4 *s4, bool into_facc) {
  CoulArgs a;
  a.s4 = s4;
  a.qd = c.cqd;
  a.cell_start = c.ccell_start;
  a.map = c.cmap;
  a.nq = c.Nq;
  a.grid = c.grid;
  a.pc = c.pc;  // the default +-1e-5 band covers an r^2 from exact integer displacements
  a.F = c.F; a.Fd = c.Fd; a.Fstride = c.N;
  a.epart = c.epart + c.off_coul;
  a.comp = c.precision == RBE_FP32_COMP;
  const double rr = c.rc * (1.0 + 1e-5) + 8.0 * std::ldexp(1.0, -24) * std::max(c.box[0], std::max(c.box[1], c.box[2]));
  a.reach2 = (float)(rr * rr);
  a.facc = into_facc ? c.facc : nullptr;
  a.fscale = (float)kFixScale32;
  a.fscale_d = kFixScale64;
  a.err = c.err;
  const dim3 g((unsigned)c.n_coul_blk), b(kCoulWarps * 32);  // every slot of the partial range
  // (per replica in a batch, like the other pair kernels)
  if (c.precision == RBE_FP64)
    return dispatch(c, coul_kernel<double>, nullptr, g, b, 0, a, true);
  return dispatch(c, coul_kernel<float>, nullptr, g, b, 0, a, true);
}

}  // namespace rbe
