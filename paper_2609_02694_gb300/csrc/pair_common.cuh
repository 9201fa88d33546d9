// pair_common.cuh -- pair interaction of the real-space part (Eqs. F_i, G_short, LJ) shared
// by the cell-list kernel and the random batch list kernel.
#pragma once
#include <cuda_fp16.h>

#include "rbe_internal.cuh"

namespace rbe {

constexpr int kPairWarps = 1;  // one-warp blocks: a finished warp frees its slot at once

struct PairArgs {
  PairSet set;
  Grid grid;
  PairConst pc;
  // single-type LJ coefficients (as in LJTable)
  float ljA, ljB, ljA12, ljB6;
  double ljAd, ljBd, ljA12d, ljB6d;
  const LJTable *table;  // device copy, multi-type only
  float *F;
  double *Fd;
  int64_t Fstride;   // N of the force arrays (SoA stride)
  int accumulate;    // add to F instead of overwriting
  double *epart;     // per-block partials (NQ_PAIR doubles each)
  int32_t *nbr;      // per-particle neighbour counts (sorted order of the set), nullable
  // Coarse-test frame: coordinates relative to the group leader are a valid minimum
  // image only while (distance of a member from the leader) + r_c < L/2 on every axis.
  // A group spans at most `smax` cells in x (one cell in y and z); boxes too small for
  // even one cell use the wrapping variant, which folds every difference into [-L/2, L/2).
  int smax;
  int trim;           // cut each row's run to the group's x-reach (rows are sorted by x)
  float L[3], invL[3];
  int comp;  // compensated (Kahan) Coulomb energy and virial sums
  // Packed half-precision candidate test: frame coordinates scaled by scale16 = 8 / r_c
  // (the cutoff maps to 8), compared with thr16 = 66.5 > 64 + the worst rounding of the
  // test (2.06 for |coordinate| < 64 scaled units, which smax16 guarantees). No true
  // neighbour is rejected; the exact decision is taken again when the pair is evaluated.
  float scale16;
  int smax16;
  // Verlet-list build (the cell kernel's BUILD variant): pc's cutoff fields then hold
  // r_list = r_c + skin, and every j != i with r_ij^2 <= r_list^2 (1 + 1e-5) in FP32 is
  // appended to i's list: warp-interleaved, entry t of the particle in slot i at
  // list[((i / 32) * K + t) * 32 + i % 32].
  int32_t *list, *len;
  int K;
  const int32_t *gate;   // build only when *gate != 0
  int32_t *maxlen;       // longest list (atomic max)
  int *err;
};

// Fold a coordinate difference into [-L/2, L/2) (only the small-box variants use it).
__device__ __forceinline__ float fold(float d, float L, float invL) {
  return mad(-L, rintf(d * invL), d);
}

template <typename real>
struct PairAcc {
  real fx, fy, fz, ulj, wlj, uc, wc;
  real cuc, cwc;  // Kahan compensations of uc, wc (compensated form)
  int nbr;
};

template <typename real>
__device__ __forceinline__ void kahan_add(real &s, real &c, real x) {
  const real y = x - c;
  const real t = s + y;
  c = (t - s) - y;
  s = t;
}

// Squared distance of the exact cutoff decision (the oracle's definition): dx_d =
// (int32)(s_i - s_j) * (L_d / 2^32) and r2 = dx^2 + dy^2 + dz^2 in FP64, no FMA.
__device__ __forceinline__ double exact_r2(const PairConst &pc, int dsx, int dsy, int dsz) {
  const double ex = __dmul_rn((double)dsx, pc.hd[0]);
  const double ey = __dmul_rn((double)dsy, pc.hd[1]);
  const double ez = __dmul_rn((double)dsz, pc.hd[2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
}

// LJ terms of one pair from 1/r^2 (types ti, tj): force factor gl (F_i = gl (r_i - r_j)),
// energy u = A r^-12 - B r^-6 and virial w = gl r^2 = r^-6 (12 A r^-6 - 6 B). With
// 1/r^2 = 0 all three are exact zeros.
template <typename real, bool MULTI>
__device__ __forceinline__ void lj_terms(const PairArgs &a, const LJTable *tab, int ti, int tj,
                                         real ir2, real &gl, real &u, real &w) {
  real A, B, A12, B6;
  if (MULTI) {
    const int pt = ti * tab->nt + tj;
    if (sizeof(real) == 8) { A = (real)tab->Ad[pt]; B = (real)tab->Bd[pt]; A12 = (real)tab->A12d[pt]; B6 = (real)tab->B6d[pt]; }
    else { A = (real)tab->A[pt]; B = (real)tab->B[pt]; A12 = (real)tab->A12[pt]; B6 = (real)tab->B6[pt]; }
  } else {
    if (sizeof(real) == 8) { A = (real)a.ljAd; B = (real)a.ljBd; A12 = (real)a.ljA12d; B6 = (real)a.ljB6d; }
    else { A = (real)a.ljA; B = (real)a.ljB; A12 = (real)a.ljA12; B6 = (real)a.ljB6; }
  }
  const real ir6 = ir2 * ir2 * ir2;
  w = ir6 * mad(A12, ir6, -B6);
  gl = w * ir2;
  u = ir6 * mad(A, ir6, -B);
}

// Pair force, energies and virial of one pair that is inside the cutoff (Eqs. F_i,
// G_short, LJ), added to acc.
template <typename real, bool LJ, bool COUL, bool MULTI>
__device__ __forceinline__ void pair_force_v(const PairArgs &a, const LJTable *tab, real dx,
                                             real dy, real dz, real r2, real qi, int ti,
                                             real qj, int tj, PairAcc<real> &acc) {
  const PairConst &pc = a.pc;
  real g = (real)0;
  if (LJ) {
    real ir2;
    if (sizeof(real) == 8) ir2 = (real)(1.0 / (double)r2);
    else ir2 = (real)__fdividef(1.0f, (float)r2);  // fast reciprocal (2 ulp)
    real gl, u, w;
    lj_terms<real, MULTI>(a, tab, ti, tj, ir2, gl, u, w);
    g += gl;
    acc.ulj += u;
    acc.wlj += w;
  }
  if (COUL) {
    const real qq = qi * qj;
    if (qq != (real)0) {
      real r, rinv, erfcv, expv;
      if (sizeof(real) == 8) {
        r = (real)sqrt((double)r2);
        rinv = (real)1 / r;
        erfcv = (real)erfc(pc.sqrt_alpha_d * (double)r);
        expv = (real)exp(-pc.alpha_d * (double)r2);
      } else {
        rinv = (real)rsqrtf((float)r2);  // 1/r and r from one reciprocal square root
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
      // erfc-Coulomb pair energies of both signs cancel heavily: compensate the sums
      if (a.comp) {
        kahan_add(acc.uc, acc.cuc, Cqq * erfcv * rinv);
        kahan_add(acc.wc, acc.cwc, gc * r2);
      } else {
        acc.uc = mad(Cqq * erfcv, rinv, acc.uc);
        acc.wc = mad(gc, r2, acc.wc);
      }
    }
  }
  acc.fx = mad(g, dx, acc.fx);
  acc.fy = mad(g, dy, acc.fy);
  acc.fz = mad(g, dz, acc.fz);
}

// Same, with the charge and type of j read from the set.
template <typename real, bool LJ, bool COUL, bool MULTI>
__device__ __forceinline__ void pair_force(const PairArgs &a, const LJTable *tab, real dx,
                                           real dy, real dz, real r2, real qi, int ti,
                                           int64_t j, PairAcc<real> &acc) {
  real qj = (real)0;
  if (COUL) qj = sizeof(real) == 8 ? (real)a.set.qd[j] : (real)a.set.qf[j];
  const int tj = MULTI ? a.set.type[j] : 0;
  pair_force_v<real, LJ, COUL, MULTI>(a, tab, dx, dy, dz, r2, qi, ti, qj, tj, acc);
}

// Branch-light evaluation for the cell-list kernel: `act` says whether this lane holds a
// candidate pair at all (idle lanes compute a masked dummy). The cutoff decision is exact:
// FP32 outside the +-1e-5 band around r_c^2, the oracle's FP64 expression inside it (a
// rare, divergent branch); in the FP64 form always the FP64 expression. A zero
// displacement (the particle itself; r^2 = 0 exactly when the integer displacement is 0)
// is never a pair. Rejected and idle lanes evaluate with 1/r^2 = 0, which makes every LJ
// term an exact zero, so no early return diverges the warp.
template <typename real, bool LJ, bool COUL, bool MULTI>
__device__ __forceinline__ void pair_eval_masked(const PairArgs &a, const LJTable *tab,
                                                 bool act, int dsx, int dsy, int dsz, real qi,
                                                 int ti, real qj, int tj,
                                                 PairAcc<real> &acc) {
  const PairConst &pc = a.pc;
  real dx, dy, dz, r2;
  bool inside;
  if (sizeof(real) == 8) {
    dx = (real)__dmul_rn((double)dsx, pc.hd[0]);
    dy = (real)__dmul_rn((double)dsy, pc.hd[1]);
    dz = (real)__dmul_rn((double)dsz, pc.hd[2]);
    r2 = (real)__dadd_rn(__dadd_rn(__dmul_rn((double)dx, (double)dx),
                                   __dmul_rn((double)dy, (double)dy)),
                         __dmul_rn((double)dz, (double)dz));
    inside = act && (double)r2 <= pc.rc2d && (double)r2 > 0.0;
  } else {
    dx = (real)((float)dsx * pc.h[0]);
    dy = (real)((float)dsy * pc.h[1]);
    dz = (real)((float)dsz * pc.h[2]);
    r2 = mad(dx, dx, mad(dy, dy, dz * dz));
    inside = act && (float)r2 < pc.rc2_lo && (float)r2 > 0.f;
    const bool band = act && (float)r2 >= pc.rc2_lo && (float)r2 <= pc.rc2_hi;
    if (band) inside = exact_r2(pc, dsx, dsy, dsz) <= pc.rc2d;
  }
  acc.nbr += inside ? 1 : 0;
  // off the pair: 1/r^2 = 0 exactly (FP64: 1/inf; FP32: the fast quotient is documented
  // to return 0 for divisors between 2^126 and 2^128)
  const real r2s = inside ? r2 : (sizeof(real) == 8 ? (real)__longlong_as_double(0x7ff0000000000000ll)
                                                    : (real)1e38f);
  real g = (real)0;
  if (LJ) {
    real ir2;
    if (sizeof(real) == 8) ir2 = (real)(1.0 / (double)r2s);
    else ir2 = (real)__fdividef(1.0f, (float)r2s);  // fast reciprocal (2 ulp)
    real gl, u, w;
    lj_terms<real, MULTI>(a, tab, ti, tj, ir2, gl, u, w);
    g += gl;
    acc.ulj += u;
    acc.wlj += w;
  }
  if (COUL) {
    const real qq = qi * qj;
    if (inside && qq != (real)0) {
      real r, rinv, erfcv, expv;
      if (sizeof(real) == 8) {
        r = (real)sqrt((double)r2);
        rinv = (real)1 / r;
        erfcv = (real)erfc(pc.sqrt_alpha_d * (double)r);
        expv = (real)exp(-pc.alpha_d * (double)r2);
      } else {
        rinv = (real)rsqrtf((float)r2);  // 1/r and r from one reciprocal square root
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
  acc.fx = mad(g, dx, acc.fx);
  acc.fy = mad(g, dy, acc.fy);
  acc.fz = mad(g, dz, acc.fz);
}

// Exact cutoff decision from the integer displacement ds = s_i - s_j (mod 2^32, the
// minimum image), then the pair force. FP32 decides outside the +-1e-5 band around r_c^2;
// inside it (and always in the FP64 form) the oracle's FP64 expression decides.
template <typename real, bool LJ, bool COUL, bool MULTI>
__device__ __forceinline__ void pair_body_ds(const PairArgs &a, const LJTable *tab, int dsx,
                                             int dsy, int dsz, real qi, int ti, real qj,
                                             int tj, PairAcc<real> &acc) {
  const PairConst &pc = a.pc;
  real dx, dy, dz, r2;
  if (sizeof(real) == 8) {
    dx = (real)__dmul_rn((double)dsx, pc.hd[0]);
    dy = (real)__dmul_rn((double)dsy, pc.hd[1]);
    dz = (real)__dmul_rn((double)dsz, pc.hd[2]);
    r2 = (real)__dadd_rn(__dadd_rn(__dmul_rn((double)dx, (double)dx),
                                   __dmul_rn((double)dy, (double)dy)),
                         __dmul_rn((double)dz, (double)dz));
    if (!((double)r2 <= pc.rc2d)) return;
  } else {
    dx = (real)((float)dsx * pc.h[0]);
    dy = (real)((float)dsy * pc.h[1]);
    dz = (real)((float)dsz * pc.h[2]);
    r2 = mad(dx, dx, mad(dy, dy, dz * dz));
    if ((float)r2 > pc.rc2_hi) return;
    if ((float)r2 >= pc.rc2_lo && !(exact_r2(pc, dsx, dsy, dsz) <= pc.rc2d)) return;
  }
  acc.nbr += 1;
  pair_force_v<real, LJ, COUL, MULTI>(a, tab, dx, dy, dz, r2, qi, ti, qj, tj, acc);
}


// Exact cutoff decision at r_c followed by the pair force (cell-list real space).
template <typename real, bool LJ, bool COUL, bool MULTI>
__device__ __forceinline__ void pair_body(const PairArgs &a, const LJTable *tab, uint32_t sxi,
                                          uint32_t syi, uint32_t szi, real qi, int ti,
                                          int64_t j, PairAcc<real> &acc) {
  const PairConst &pc = a.pc;
  const int dsx = (int)(sxi - a.set.sx[j]);
  const int dsy = (int)(syi - a.set.sy[j]);
  const int dsz = (int)(szi - a.set.sz[j]);
  real dx, dy, dz, r2;
  if (sizeof(real) == 8) {
    dx = (real)__dmul_rn((double)dsx, pc.hd[0]);
    dy = (real)__dmul_rn((double)dsy, pc.hd[1]);
    dz = (real)__dmul_rn((double)dsz, pc.hd[2]);
    r2 = (real)__dadd_rn(__dadd_rn(__dmul_rn((double)dx, (double)dx),
                                   __dmul_rn((double)dy, (double)dy)),
                         __dmul_rn((double)dz, (double)dz));
    if (!((double)r2 <= pc.rc2d)) return;
  } else {
    dx = (real)((float)dsx * pc.h[0]);
    dy = (real)((float)dsy * pc.h[1]);
    dz = (real)((float)dsz * pc.h[2]);
    r2 = mad(dx, dx, mad(dy, dy, dz * dz));
    if ((float)r2 > pc.rc2_hi) return;
    if ((float)r2 >= pc.rc2_lo) {  // exact decision inside the band
      if (!(exact_r2(pc, dsx, dsy, dsz) <= pc.rc2d)) return;
    }
  }
  acc.nbr += 1;
  pair_force<real, LJ, COUL, MULTI>(a, tab, dx, dy, dz, r2, qi, ti, j, acc);
}

}  // namespace rbe
