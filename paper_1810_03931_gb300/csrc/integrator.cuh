// integrator.cuh -- the per-thread integrator kernel (one independent ODE
// system per thread, Sec. 6.1/6.4 of the paper) for both schemes of Sec. 3,
// with the event handling of Sec. 4 / 6.6, the accessories of Sec. 5 / 6.7 and
// the initialization / finalization hooks of Sec. 6.8.
//
// GB300 design
//  * The state of a system lives in registers for the whole launch; a launch
//    runs many consecutive slices (the iterated Solve of Sec. 7.1.1) so the
//    state never round-trips through HBM between slices.
//  * Every loop iteration is ONE trial Runge-Kutta step per lane.  A lane
//    that is locating an event (bracketed root search in the step size, re-stepping from
//    the last accepted point) takes its trial step through the same stage
//    code as the lanes that take normal steps, so adaptive divergence, event
//    location and slice / system changes of single lanes never serialise the
//    warp's FP64 work; the bookkeeping branches are short.
//  * The warp leaves the loop only when no lane has work (warp vote).
//  * Persistent launches refill a lane from a device work queue (atomic
//    counter) the moment its system finishes.
//  * Runge-Kutta coefficients are compile-time immediates; per-solver
//    properties come from the kernel parameter block.
#pragma once

#include <cooperative_groups.h>

#include "bits.cuh"
#include "common.cuh"
#include "models.cuh"

namespace odegpu {

// ---- Butcher tableaux ------------------------------------------------------
// Cash & Karp (ACM TOMS 16, 1990), embedded 4(5) pair; the fifth-order
// solution is propagated and E = b5 - b4 weighs the error estimate.
namespace ck {
constexpr double c2 = 1.0 / 5.0, c3 = 3.0 / 10.0, c4 = 3.0 / 5.0, c5 = 1.0, c6 = 7.0 / 8.0;
constexpr double a21 = 1.0 / 5.0;
constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
constexpr double a41 = 3.0 / 10.0, a42 = -9.0 / 10.0, a43 = 6.0 / 5.0;
constexpr double a51 = -11.0 / 54.0, a52 = 5.0 / 2.0, a53 = -70.0 / 27.0, a54 = 35.0 / 27.0;
constexpr double a61 = 1631.0 / 55296.0, a62 = 175.0 / 512.0, a63 = 575.0 / 13824.0,
                 a64 = 44275.0 / 110592.0, a65 = 253.0 / 4096.0;
constexpr double b1 = 37.0 / 378.0, b3 = 250.0 / 621.0, b4 = 125.0 / 594.0, b6 = 512.0 / 1771.0;
constexpr double bs1 = 2825.0 / 27648.0, bs3 = 18575.0 / 48384.0, bs4 = 13525.0 / 55296.0,
                 bs5 = 277.0 / 14336.0, bs6 = 1.0 / 4.0;
constexpr double e1 = b1 - bs1, e3 = b3 - bs3, e4 = b4 - bs4, e5 = 0.0 - bs5, e6 = b6 - bs6;
}  // namespace ck

template <int PREC>
struct StageType { using type = double; };
template <>
struct StageType<kFP32RHS> { using type = float; };

// ---- harmonic forcing ------------------------------------------------------
// For a stage at t + c h the forcing angle advances by c x with x = omega h.
// For |x| <= kSmallAngle = 0.1, cos(c x) and sin(c x) / x are cubics in
// U = x^2 with the powers of c folded into compile-time coefficients: the
// Taylor series to U^4 (a_k = (-1)^k c^2k / (2k)!, b_k = (-1)^k c^(2k+1) /
// (2k+1)!; the U^5 terms are below 3e-17) with its U^4 term replaced by the
// best cubic approximation of U^4 on one of two intervals, [0, U1] and
// [U1, kSmallAngle^2] with U1 = 0.07^2 (Chebyshev economization, Lanczos):
// on [m - w, m + w], U^4 = r(U) + (w^4 / 8) T4((U - m) / w) with
//   r(U) = 4 m U^3 + (w^2 - 6 m^2) U^2 + (4 m^3 - 2 m w^2) U
//          + m^2 w^2 - m^4 - w^4 / 8,
// so the replacement adds at most |a4| w^4 / 8 (1.3e-16 for cos at c = 1).
// The interval is chosen per lane by selecting coefficients (no branch).
// Larger angles call sincos.
constexpr double kSmallAngle = 0.1;
constexpr double kU1 = 0.07 * 0.07;

__host__ __device__ constexpr double cpow(double c, int k) { return k == 0 ? 1.0 : c * cpow(c, k - 1); }
__host__ __device__ constexpr double fact(int k) { return k <= 1 ? 1.0 : k * fact(k - 1); }
__host__ __device__ constexpr double cos_coef(double c, int k) { return (k % 2 ? -1.0 : 1.0) * cpow(c, 2 * k) / fact(2 * k); }
__host__ __device__ constexpr double sin_coef(double c, int k) {
  return (k % 2 ? -1.0 : 1.0) * cpow(c, 2 * k + 1) / fact(2 * k + 1);
}
// coefficient j (0..3) of the cubic economized from the quartic with U^j
// coefficient aj and U^4 coefficient a4 on [m - w, m + w]
__host__ __device__ constexpr double econ3(double aj, double a4, int j, double m, double w) {
  return j == 3 ? aj + a4 * 4.0 * m
       : j == 2 ? aj + a4 * (w * w - 6.0 * m * m)
       : j == 1 ? aj + a4 * (4.0 * m * m * m - 2.0 * m * w * w)
                : aj + a4 * (m * m * w * w - cpow(m, 4) - cpow(w, 4) / 8.0);
}

// Coefficients of cos(c x) (a0..a3) and sin(c x) / x (b0..b3) on interval I
// (0: [0, U1], 1: [U1, kSmallAngle^2]).
template <int CNUM, int CDEN, int I>
struct AngleCubic {
  static constexpr double c = (double)CNUM / (double)CDEN;
  static constexpr double lo = I == 0 ? 0.0 : kU1, hi = I == 0 ? kU1 : kSmallAngle * kSmallAngle;
  static constexpr double m = 0.5 * (lo + hi), w = 0.5 * (hi - lo);
  static constexpr double a4 = cos_coef(c, 4), b4 = sin_coef(c, 4);
  static constexpr double a0 = econ3(1.0, a4, 0, m, w), a1 = econ3(cos_coef(c, 1), a4, 1, m, w),
                          a2 = econ3(cos_coef(c, 2), a4, 2, m, w), a3 = econ3(cos_coef(c, 3), a4, 3, m, w);
  static constexpr double b0 = econ3(sin_coef(c, 0), b4, 0, m, w), b1 = econ3(sin_coef(c, 1), b4, 1, m, w),
                          b2 = econ3(sin_coef(c, 2), b4, 2, m, w), b3 = econ3(sin_coef(c, 3), b4, 3, m, w);
};

// cd = cos(c x), sd = sin(c x) for |x| <= kSmallAngle; lo: U <= U1
template <int CNUM, int CDEN>
__device__ __forceinline__ void small_angle_c(double x, double U, bool lo, double& cd, double& sd) {
  using L = AngleCubic<CNUM, CDEN, 0>;
  using H = AngleCubic<CNUM, CDEN, 1>;
  const double a3 = lo ? L::a3 : H::a3, a2 = lo ? L::a2 : H::a2, a1 = lo ? L::a1 : H::a1,
               a0 = lo ? L::a0 : H::a0;
  const double b3 = lo ? L::b3 : H::b3, b2 = lo ? L::b2 : H::b2, b1 = lo ? L::b1 : H::b1,
               b0 = lo ? L::b0 : H::b0;
  cd = fma(fma(fma(U, a3, a2), U, a1), U, a0);
  sd = x * fma(fma(fma(U, b3, b2), U, b1), U, b0);
}

// (sin, cos)(a) in binary32 for a binary64 angle a: a is reduced to
// r = a - k pi/2 in [-pi/4, pi/4] in binary64 (k = rint(a 2/pi) by adding
// 1.5 * 2^52, whose low mantissa bits then hold k mod 4), r is rounded once,
// and the Taylor series of sin and cos at 0 up to r^9 / 9! and r^10 / 10!
// (first omitted terms below 2e-10) are evaluated in binary32; the quadrant
// k mod 4 swaps and negates them.  Valid for |a| < 2^50.
__device__ __forceinline__ void sincos_quarter(double a, float& s, float& c) {
  constexpr double kShift = 6755399441055744.0;  // 1.5 * 2^52
  const double ks = fma(a, 2.0 / CUDART_PI, kShift);
  const int q = __double2loint(ks) & 3;
  const float r = (float)fma(-(ks - kShift), 0.5 * CUDART_PI, a);
  const float r2 = r * r;
  // coefficients as compile-time constants
  constexpr float s1 = (float)sin_coef(1.0, 1), s2 = (float)sin_coef(1.0, 2), s3 = (float)sin_coef(1.0, 3),
                  s4 = (float)sin_coef(1.0, 4);
  constexpr float c1 = (float)cos_coef(1.0, 1), c2 = (float)cos_coef(1.0, 2), c3 = (float)cos_coef(1.0, 3),
                  c4 = (float)cos_coef(1.0, 4), c5 = (float)cos_coef(1.0, 5);
  const float sr = r * fmaf(fmaf(fmaf(fmaf(r2, s4, s3), r2, s2), r2, s1), r2, 1.0f);
  const float cr = fmaf(fmaf(fmaf(fmaf(fmaf(r2, c5, c4), r2, c3), r2, c2), r2, c1), r2, 1.0f);
  const float ns = -sr, nc = -cr;
  s = (q == 0) ? sr : (q == 1) ? cr : (q == 2) ? ns : nc;
  c = (q == 0) ? cr : (q == 1) ? ns : (q == 2) ? nc : sr;
}

// Binary32 rotation factors for the angle c x, |x| <= 0.1: Taylor series in
// U = x^2 up to U^2 (first omitted terms below 1.4e-9).
template <int CNUM, int CDEN>
__device__ __forceinline__ void small_angle_f(float x, float U, float& cd, float& sd) {
  constexpr double c = (double)CNUM / (double)CDEN;
  constexpr float a1 = (float)cos_coef(c, 1), a2 = (float)cos_coef(c, 2);
  constexpr float b0 = (float)sin_coef(c, 0), b1 = (float)sin_coef(c, 1), b2 = (float)sin_coef(c, 2);
  cd = fmaf(fmaf(U, a2, a1), U, 1.0f);
  sd = x * fmaf(fmaf(U, b2, b1), U, b0);
}

// (sin, cos)(omega t) of the harmonic forcing.  A model whose forcing
// frequency is one period per unit time (omega = 2 pi: Keller-Miksis in its
// time tau) takes sincospi(2 t), whose argument reduction is exact, instead
// of rounding 2 pi t first.
template <class M>
__device__ __forceinline__ void forcing_sincos(double w, double t, double& s, double& c) {
  if constexpr (M::kUnitPeriodForcing) {
    (void)w;
    sincospi(2.0 * t, &s, &c);
  } else {
    sincos(w * t, &s, &c);
  }
}

// ---- one trial step --------------------------------------------------------
// From (t, y) with step hs and the cached first stage k1 = f(t, y), compute
// the new state ynew and (RKCK45) the error estimate err = hs * sum e_i k_i.
// Stage states and f are in precision T; ynew and err are binary64.
// Harmonic forcing in binary64: (C, S) = (cos, sin)(omega t) at the lane's t;
// a stage at t + c hs gets (cos, sin)(omega (t + c hs)) by angle addition with
// d = omega c hs, and the c = 1 stage returns them in (Cn, Sn) as the anchor
// of the next step.  Large d (long steps) falls back to sincos.
// Harmonic forcing in binary32: the anchor (C, S) = (cos, sin)(omega t) comes
// from sincos_quarter (binary64 reduction of omega t, binary32 series) once
// per accepted step, and a stage rotates it by c omega hs in binary32.
// Rounding t itself to binary32 would put an error of ulp(t) / 2 into the
// phase (2.4e-4 rad at t = 7000).
template <class M, int SCHEME, int PREC>
struct Stepper {
  static constexpr int n = M::N, P = M::P;
  using T = typename StageType<PREC>::type;
  static constexpr bool kRotate = (PREC == kFP64) && (M::kForcing != kNoForcing);

  // Stage time t + c hs with c = CNUM / CDEN; in binary64 the forcing
  // (cos, sin)(omega (t + c hs)) follows from the anchor (C, S) by angle
  // addition when |omega hs| <= 0.1 (x = omega hs, U = x^2 precomputed).
  template <int CNUM, int CDEN>
  static __device__ __forceinline__ Stage<T> stage_at(double t, double hs, T tb, T h,
                                                      const T (&mct)[3], T C, T S, double w,
                                                      double x, double U, bool small, bool lo,
                                                      T xw) {
    constexpr double c = (double)CNUM / (double)CDEN;
    Stage<T> st;
    if constexpr (kRotate) {
      st.t = t + c * hs;
      if (small) {
        double cd, sd;
        small_angle_c<CNUM, CDEN>(x, U, lo, cd, sd);
        st.c = C * cd - S * sd;
        st.s = S * cd + C * sd;
      } else {
        forcing_sincos<M>(w, st.t, st.s, st.c);
      }
    } else {
      (void)mct; (void)U; (void)lo;
      st.t = tb + (T)c * h;
      if constexpr (M::kForcing != kNoForcing) {
        if (small) {
          T cd, sd;
          small_angle_f<CNUM, CDEN>(xw, xw * xw, cd, sd);
          st.c = C * cd - S * sd;
          st.s = S * cd + C * sd;
        } else {
          sincos_quarter(fma(c, w * hs, w * t), st.s, st.c);
        }
      } else {
        (void)t; (void)hs; (void)C; (void)S; (void)w; (void)x; (void)small; (void)lo; (void)xw;
        st.c = st.s = (T)0;
      }
    }
    return st;
  }

  // yb: the state y in precision T (y itself in binary64).  tab (RK4 only, or
  // null): (cos, sin) of omega t at the half-step grid of the slice, the
  // stages at t + hs / 2 and t + hs being entries tab[1] and tab[2].
  static __device__ __forceinline__ void step(double t, const double (&y)[n], const T (&yb)[n],
                                              double hs, const T (&pt)[P], const T (&mct)[3],
                                              const T (&k1)[n], T C, T S, double w,
                                              double (&ynew)[n], double (&err)[n], double& Cn,
                                              double& Sn, const double2* tab = nullptr) {
    const T h = (T)hs;
    const T tb = (T)t;
    const double x = w * hs, U = x * x;
    const bool small = fabs(x) <= kSmallAngle;
    const bool lo = dbits(U) <= dbits(kU1);  // U >= 0: compared on the integer pipe
    const T xw = (!kRotate && M::kForcing != kNoForcing) ? (T)x : (T)0;
    T ys[n];
    if constexpr (SCHEME == kRKCK45) {
      using namespace ck;
      T k2[n], k3[n], k4[n], k5[n], k6[n];
#pragma unroll
      for (int m = 0; m < n; m++) ys[m] = stage(y[m], yb[m], hs, h, (T)a21 * k1[m]);
      M::template rhs<T>(stage_at<1, 5>(t, hs, tb, h, mct, C, S, w, x, U, small, lo, xw), ys, pt, mct, k2);
#pragma unroll
      for (int m = 0; m < n; m++) ys[m] = stage(y[m], yb[m], hs, h, (T)a31 * k1[m] + (T)a32 * k2[m]);
      M::template rhs<T>(stage_at<3, 10>(t, hs, tb, h, mct, C, S, w, x, U, small, lo, xw), ys, pt, mct, k3);
#pragma unroll
      for (int m = 0; m < n; m++)
        ys[m] = stage(y[m], yb[m], hs, h, (T)a41 * k1[m] + (T)a42 * k2[m] + (T)a43 * k3[m]);
      M::template rhs<T>(stage_at<3, 5>(t, hs, tb, h, mct, C, S, w, x, U, small, lo, xw), ys, pt, mct, k4);
#pragma unroll
      for (int m = 0; m < n; m++)
        ys[m] = stage(y[m], yb[m], hs, h,
                      (T)a51 * k1[m] + (T)a52 * k2[m] + (T)a53 * k3[m] + (T)a54 * k4[m]);
      const Stage<T> s5 = stage_at<1, 1>(t, hs, tb, h, mct, C, S, w, x, U, small, lo, xw);
      M::template rhs<T>(s5, ys, pt, mct, k5);
      Cn = (double)s5.c;
      Sn = (double)s5.s;
#pragma unroll
      for (int m = 0; m < n; m++)
        ys[m] = stage(y[m], yb[m], hs, h,
                      (T)a61 * k1[m] + (T)a62 * k2[m] + (T)a63 * k3[m] + (T)a64 * k4[m] +
                          (T)a65 * k5[m]);
      M::template rhs<T>(stage_at<7, 8>(t, hs, tb, h, mct, C, S, w, x, U, small, lo, xw), ys, pt, mct, k6);
#pragma unroll
      for (int m = 0; m < n; m++) {
        // binary64 state update and error estimate; with binary32 stages the
        // weighted stage sums are formed in binary32 (the stages carry that
        // rounding already) and promoted once
        const T sb = (T)b1 * k1[m] + (T)b3 * k3[m] + (T)b4 * k4[m] + (T)b6 * k6[m];
        ynew[m] = y[m] + hs * (double)sb;
        const T se = (T)e1 * k1[m] + (T)e3 * k3[m] + (T)e4 * k4[m] + (T)e5 * k5[m] + (T)e6 * k6[m];
        err[m] = hs * (double)se;
      }
    } else {
      T k2[n], k3[n], k4[n];
      const T half = (T)0.5;
      Stage<T> sh, s4;
      if (kRotate && tab != nullptr) {
        const double2 f1 = tab[1], f2 = tab[2];
        sh.t = t + 0.5 * hs; sh.c = f1.x; sh.s = f1.y;
        s4.t = t + hs; s4.c = f2.x; s4.s = f2.y;
      } else {
        sh = stage_at<1, 2>(t, hs, tb, h, mct, C, S, w, x, U, small, lo, xw);
        s4 = stage_at<1, 1>(t, hs, tb, h, mct, C, S, w, x, U, small, lo, xw);
      }
#pragma unroll
      for (int m = 0; m < n; m++) ys[m] = stage(y[m], yb[m], hs, h, half * k1[m]);
      M::template rhs<T>(sh, ys, pt, mct, k2);
#pragma unroll
      for (int m = 0; m < n; m++) ys[m] = stage(y[m], yb[m], hs, h, half * k2[m]);
      M::template rhs<T>(sh, ys, pt, mct, k3);
#pragma unroll
      for (int m = 0; m < n; m++) ys[m] = stage(y[m], yb[m], hs, h, k3[m]);
      M::template rhs<T>(s4, ys, pt, mct, k4);
      Cn = (double)s4.c;
      Sn = (double)s4.s;
#pragma unroll
      for (int m = 0; m < n; m++) {
        const T sb = (T)(1.0 / 6.0) * k1[m] + (T)(1.0 / 3.0) * k2[m] + (T)(1.0 / 3.0) * k3[m] +
                     (T)(1.0 / 6.0) * k4[m];
        ynew[m] = y[m] + hs * (double)sb;
        err[m] = 0.0;
      }
    }
  }

  // Stage state y + h * s: binary64 when T is double, binary32 otherwise.
  static __device__ __forceinline__ T stage(double y, T yb, double hs, T h, T s) {
    if constexpr (PREC == kFP64) {
      (void)yb; (void)h;
      return y + hs * s;
    } else {
      (void)y; (void)hs;
      return yb + h * s;
    }
  }
};

// x^(-1/5) for x within the clamping range of the step-size factor: a
// binary32 seed (relative error ~2e-7) refined by one Newton step for
// z^-5 = x in binary64, z <- z + z (1 - x z^5) / 5, which squares the error
// to ~2e-13 -- far below the rounding noise of the error estimate itself
// (the estimate is a difference of nearly equal sums).  Six binary64
// operations instead of a general pow().
__device__ __forceinline__ double rpow_fifth(double x) {
  const double z = (double)exp2f(-0.2f * __log2f((float)x));
  const double z2 = z * z;
  const double r = fma(-x, z2 * z2 * z, 1.0);
  return fma(0.2 * z, r, z);
}

// Root in (0, 1) of the cubic Hermite interpolant of F over one step from its
// end values F0, F1 (opposite signs) and end slopes D0, D1 (dF/dt times the
// step): three Newton steps from the secant root, kept inside [0, 1].
__device__ __forceinline__ double hermite_root(double F0, double F1, double D0, double D1) {
  double s = F0 / (F0 - F1);
#pragma unroll
  for (int it = 0; it < 3; it++) {
    const double u = 1.0 - s;
    const double h00 = (1.0 + 2.0 * s) * u * u, h10 = s * u * u;
    const double h01 = s * s * (3.0 - 2.0 * s), h11 = s * s * (s - 1.0);
    const double H = h00 * F0 + h10 * D0 + h01 * F1 + h11 * D1;
    const double dH = (6.0 * s * s - 6.0 * s) * (F0 - F1) + (3.0 * s * s - 4.0 * s + 1.0) * D0 +
                      (3.0 * s * s - 2.0 * s) * D1;
    if (dH != 0.0) s -= H / dH;
    s = fmin(fmax(s, 0.0), 1.0);
  }
  return s;
}

// Is event j crossed in its allowed direction between F_old (outside the
// zone) and F_new?  Landing inside the zone counts (Sec. 4, MATLAB direction
// rule of Sec. 6.6).
__device__ __forceinline__ bool crossed(const Props& pr, int j, double F_old, double F_new) {
  const double tol = pr.evt_tol[j];
  const bool down = dpos(F_old) && dle(F_new, tol);
  const bool up = dneg(F_old) && dle(-tol, F_new);
  const int dir = pr.evt_dir[j];
  return dir < 0 ? down : (dir > 0 ? up : (down || up));
}

// ---- the per-lane state machine -------------------------------------------
template <class M, int SCHEME, int PREC>
struct Lane {
  static constexpr int n = M::N, P = M::P, A = M::A, E = M::E;
  using T = typename StageType<PREC>::type;
  using St = Stepper<M, SCHEME, PREC>;

  int sys;
  int slice;
  int my_slices;
  int left0;  // served slots: the slice budget loaded with the slot
  int status;
  bool k1ok;
  bool locating;
  int jstar;
  int loc_it;
  long long steps;
  unsigned int nacc, nrej;
  double t, t0, t1, h, hnext;
  double y[n];
  double p[P];
  T pt[P];
  T mct[3];
  double acc[A];
  double F[E];
  bool leaving[E];
  bool det[E];
  int inzone[E];
  int ecnt[E];
  T k1[n];
  double lo, hi, yhi[n];
  double theta_a, theta_b;  // narrowed bracket to verify first; in phase 2
                            // theta_a holds F_jstar at lo (F at hi follows from yhi)
  int loc_phase;            // 0: try theta_a, 1: try theta_b, 2: refine the bracket
  double fC, fS;    // cos, sin of omega t at the lane's t (binary64 forcing)
  double fCn, fSn;  // the same at t + hs of the last normal trial step
  T gC, gS;         // binary32 form: cos, sin of omega t at the lane's t
  T yt[n];          // binary32 form: the state y rounded once per accepted point
  double w;         // forcing angular frequency
  const double2* tab;  // RK4: block-shared (cos, sin) of omega t on the half-step
                       // grid of the slice time domain (tab_t0, tab_t1), or null
  int tab_n;           // steps the table covers
  double tab_t0, tab_t1;
  bool use_tab;        // this slice lies on the table's grid

  // Load the slot; false when the system has no slice to run in this launch.
  // CG: load through L2 only (ld.global.cg), for slots that other agents (the
  // host's copies, other SMs) may have rewritten while this kernel runs.
  template <bool CG = false>
  __device__ __forceinline__ bool load(const KArgs& a) {
    const size_t N = (size_t)a.ld;  // 64-bit component offsets
    auto ld = [](const double* q) { return CG ? __ldcg(q) : *q; };
    my_slices = a.n_slices;
    int my_slices_left = 0;
    if (a.slices_left != nullptr) {
      my_slices_left = CG ? __ldcg(a.slices_left + sys) : a.slices_left[sys];
      my_slices = min(my_slices, my_slices_left);
    }
    (void)my_slices_left;
    if (my_slices <= 0) return false;
    t0 = ld(a.td + sys);
    t1 = ld(a.td + N + sys);
#pragma unroll
    for (int m = 0; m < n; m++) y[m] = ld(a.y + m * N + sys);
#pragma unroll
    for (int m = 0; m < P; m++) {
      p[m] = ld(a.p + m * N + sys);
      pt[m] = (T)p[m];
    }
    slice = 0;
    nacc = 0;
    nrej = 0;
    if (CG) left0 = my_slices_left;
    return true;
  }

  // Store the slot.  CG: counters and the slice budget are read through L2
  // and the budget is written from the value loaded with the slot (another
  // agent may have rewritten the slot since this SM last cached it).
  template <bool CG = false>
  __device__ __forceinline__ void store(const KArgs& a) {
    const size_t N = (size_t)a.ld;  // 64-bit component offsets
    a.td[sys] = t0;
    a.td[N + sys] = t1;
#pragma unroll
    for (int m = 0; m < n; m++) a.y[m * N + sys] = y[m];
#pragma unroll
    for (int m = 0; m < A; m++) a.acc[m * N + sys] = acc[m];
    a.status[sys] = status;
#pragma unroll
    for (int j = 0; j < E; j++) a.ecnt[j * N + sys] = a.pr.events_on ? ecnt[j] : 0;
    if (CG) {
      a.nacc[sys] = __ldcg(a.nacc + sys) + nacc;
      a.nrej[sys] = __ldcg(a.nrej + sys) + nrej;
      if (a.slices_left != nullptr) a.slices_left[sys] = left0 - slice;
    } else {
      a.nacc[sys] += nacc;
      a.nrej[sys] += nrej;
      if (a.slices_left != nullptr) a.slices_left[sys] -= slice;
    }
  }

  __device__ __forceinline__ void anchor_forcing() {
    if constexpr (St::kRotate) forcing_sincos<M>(w, t, fS, fC);
  }

  // Start a slice: Initialization hook (Sec. 6.8), event state at t0 (a
  // point already inside a zone is in the leaving state and is not detected,
  // Sec. 4 / Sec. 7.2), initial step (Sec. 6.4).
  __device__ __forceinline__ void begin_slice(const KArgs& a) {
    const Props& pr = a.pr;
    t = t0;
    M::acc_init(t, y, acc);
    if (pr.events_on) {
      M::events(t, y, p, F);
#pragma unroll
      for (int j = 0; j < E; j++) {
        leaving[j] = dabs_le(F[j], pr.evt_tol[j]);
        inzone[j] = 0;
        ecnt[j] = 0;
      }
    } else {
#pragma unroll
      for (int j = 0; j < E; j++) ecnt[j] = 0;
    }
    if constexpr (SCHEME == kRK4) {
      double nsteps = ceil((t1 - t0) / a.h0 - 1e-9);
      nsteps = nsteps < 1.0 ? 1.0 : nsteps;
      h = (t1 - t0) / nsteps;
    } else {
      h = fmin(fmax(a.h0, pr.hmin), pr.hmax);
    }
    status = (t < t1) ? kStNone : kStTEnd;
    steps = 0;
    k1ok = false;
    locating = false;
    if constexpr (SCHEME == kRK4 && St::kRotate) use_tab = tab != nullptr && t0 == tab_t0 && t1 == tab_t1;
    anchor_forcing();
  }

  // End of a slice: Finalization (Sec. 6.8) -- the time-domain update and the
  // model's own hook -- and the record.
  __device__ __forceinline__ void end_slice(const KArgs& a) {
    const double t_end = t;
    if (a.pr.td_mode == kTdT0ToT) {
      t0 = t_end;
    } else if (a.pr.td_mode == kTdShift) {
      const double span = t1 - t0;
      t0 = t_end;
      t1 = t_end + span;
    }
    M::finalize(y, acc);
    if (a.records != nullptr && slice >= a.n_skip) {
      const int N = a.N;
      constexpr int R = A + n + 1;
      double* rec = a.records + (size_t)(slice - a.n_skip) * R * N + sys;
#pragma unroll
      for (int m = 0; m < A; m++) rec[(size_t)m * N] = acc[m];
#pragma unroll
      for (int m = 0; m < n; m++) rec[(size_t)(A + m) * N] = y[m];
      rec[(size_t)(A + n) * N] = t_end;
    }
    slice++;
  }

  // Accept the point (tnew, ynew) with the detected-event flags det[]:
  // ordinary accessories, then for each detected event in ascending order its
  // counter, event accessories and action, then the zone bookkeeping and the
  // stop checks (Sec. 4, 6.6, 6.7).
  __device__ __forceinline__ void accept(const Props& pr, double tnew, const double (&ynew)[n],
                                         bool last, bool located) {
    t = tnew;
    if constexpr (St::kRotate) {
      if (located) {
        // a located point is off the fixed-step grid: the table no longer applies
        if constexpr (SCHEME == kRK4) use_tab = false;
        anchor_forcing();
      } else {
        fC = fCn;
        fS = fSn;
      }
    }
#pragma unroll
    for (int m = 0; m < n; m++) y[m] = ynew[m];
    nacc++;
    if constexpr (SCHEME == kRKCK45) h = hnext;
    k1ok = false;
    M::acc_ordinary(t, y, acc);
    if (pr.events_on) {
#pragma unroll
      for (int j = 0; j < E; j++) {
        if (det[j]) {
          ecnt[j]++;
          M::acc_event(j, ecnt[j], t, y, acc);
          M::action(j, y, p);
        }
      }
      M::events(t, y, p, F);
#pragma unroll
      for (int j = 0; j < E; j++) {
        const bool in_zone = dabs_le(F[j], pr.evt_tol[j]);
        if (det[j]) {
          leaving[j] = true;
          inzone[j] = 0;
        } else if (leaving[j]) {
          if (!in_zone) {
            leaving[j] = false;
            inzone[j] = 0;
          } else {
            inzone[j]++;
            if (pr.max_eq > 0 && inzone[j] >= pr.max_eq) status = kStEquilibrium;
          }
        } else if (in_zone) {
          leaving[j] = true;
          inzone[j] = 0;
        }
      }
#pragma unroll
      for (int j = 0; j < E; j++)
        if (det[j] && pr.evt_stop[j] > 0 && ecnt[j] >= pr.evt_stop[j]) status = kStEventStop;
    }
    if (status == kStNone && last && !located) status = kStTEnd;
  }

  __device__ __forceinline__ void finish_location(const Props& pr) {
    locating = false;
    const double tnew = t + hi;
    if (E > 1) {
      double Fn[E];
      M::events(tnew, yhi, p, Fn);
#pragma unroll
      for (int j = 0; j < E; j++)
        if (j != jstar) det[j] = det[j] && crossed(pr, j, F[j], Fn[j]);
    }
    accept(pr, tnew, yhi, false, true);
  }

  // theta* for the narrowed bracket: root of the cubic Hermite interpolant of
  // event js over the step (t, t + hs) from F and dF/dt at both ends; dF/dt
  // at the end needs one right-hand side at (t + hs, ynew).  Called once per
  // located event and kept out of line so that its registers do not raise
  // the step loop's register count.
  // Arguments are scalars and a pointer: array references would make the
  // caller keep copies of its state and parameters in local memory for the
  // call (stores on every step).  The parameters are reloaded through L2
  // (pg[m * ld], the slot's column) and converted to the stage precision.
  static __device__ __noinline__ double predict_root(int js, double t, double hs, double f_old,
                                                     double f_new, double rate_old, double y0,
                                                     double y1, double y2, double y3,
                                                     const double* pg, long long ld, double mc0,
                                                     double mc1, double mc2, double Cn, double Sn,
                                                     double w) {
    const double yn[kMaxN] = {y0, y1, y2, y3};
    T yb[n], f1[n], pt[P];
    const T mct[3] = {(T)mc0, (T)mc1, (T)mc2};
#pragma unroll
    for (int m = 0; m < n; m++) yb[m] = (T)yn[m];
#pragma unroll
    for (int m = 0; m < P; m++) pt[m] = (T)__ldcg(pg + m * ld);
    Stage<T> s1;
    if constexpr (St::kRotate) {
      (void)w;
      s1.t = t + hs;
      s1.c = Cn;
      s1.s = Sn;
    } else {
      (void)Cn; (void)Sn;
      s1.t = (T)(t + hs);
      s1.c = s1.s = (T)0;
      if constexpr (M::kForcing != kNoForcing) sincos_quarter(w * (t + hs), s1.s, s1.c);
      else (void)w;
    }
    M::template rhs<T>(s1, yb, pt, mct, f1);
    return hs * hermite_root(f_old, f_new, hs * rate_old, hs * M::event_rate(js, f1));
  }

  // One trial step (normal, or a locating step inside the event's bracket).
  __device__ __forceinline__ void trial(const KArgs& a) {
    const Props& pr = a.pr;
    double hs;
    bool last = false;
    if (locating) {
      double th = 0.5 * (lo + hi);
      if (loc_phase == 0) th = theta_a;
      else if (loc_phase == 1) th = theta_b;
      if (!(th > lo && th < hi)) {
        // a verification point outside the current bracket: refine.  Before
        // the first verification lo is 0, where F is the accepted point's.
        if (loc_phase == 0) {
          theta_a = F[0];
#pragma unroll
          for (int j = 1; j < E; j++)
            if (j == jstar) theta_a = F[j];
        }
        loc_phase = 2;
        th = 0.5 * (lo + hi);
      }
      if (loc_phase == 2 && (loc_it & 3) != 3) {
        // the secant of the bracket's end values (the paper's secant
        // iteration), when it falls strictly inside; every fourth trial
        // bisects, so the bracket at least halves every four trials whatever
        // the secant does
        double Fh[E];
        M::events(t + hi, yhi, p, Fh);
        double fhi = Fh[0];
#pragma unroll
        for (int j = 1; j < E; j++)
          if (j == jstar) fhi = Fh[j];
        // (F at the two ends has opposite signs, so fhi - flo is finite and
        // nonzero; a reciprocal refined by Newton steps is exact enough for
        // a trial point, which only has to lie inside the bracket)
        const double flo = theta_a;
        const double ts = lo - flo * (hi - lo) * recip_nr(fhi - flo);
        if (ts > lo && ts < hi) th = ts;
      }
      if (!(th > lo && th < hi) || loc_it >= 200) {
        finish_location(pr);
        return;
      }
      hs = th;
    } else {
      if (steps >= pr.max_steps) {
        status = kStStepBudget;
        return;
      }
      hs = h;
      if (t1 - t <= hs * (1.0 + 1e-9)) {
        hs = t1 - t;
        last = true;
      }
    }
    if (!k1ok) {
      if constexpr (PREC != kFP64) {
        // the state in binary32, kept for the trials from this point
#pragma unroll
        for (int m = 0; m < n; m++) yt[m] = (T)y[m];
      }
      Stage<T> st0;
      if constexpr (St::kRotate) {
        st0.t = t;
        st0.c = fC;
        st0.s = fS;
        if constexpr (SCHEME == kRK4) {
          if (use_tab && !locating && steps < tab_n) {
            const double2 f0 = tab[2 * steps];
            st0.c = f0.x;
            st0.s = f0.y;
          }
        }
      } else {
        // binary32 forcing anchor at the new t, kept for the trials from t
        if constexpr (M::kForcing != kNoForcing) sincos_quarter(w * t, gS, gC);
        else gC = gS = (T)0;
        st0.t = (T)t;
        st0.c = gC;
        st0.s = gS;
      }
      if constexpr (PREC == kFP64) M::template rhs<T>(st0, y, pt, mct, k1);
      else M::template rhs<T>(st0, yt, pt, mct, k1);
      k1ok = true;
    }
    double ynew[n], err[n], Cn = 0.0, Sn = 0.0;
    if constexpr (St::kRotate) {
      const double2* tb = nullptr;
      if constexpr (SCHEME == kRK4) tb = (use_tab && !locating && steps < tab_n) ? tab + 2 * steps : nullptr;
      St::step(t, y, y, hs, pt, mct, k1, fC, fS, w, ynew, err, Cn, Sn, tb);
    }
    else if constexpr (PREC == kFP64) St::step(t, y, y, hs, pt, mct, k1, gC, gS, w, ynew, err, Cn, Sn);
    else St::step(t, y, yt, hs, pt, mct, k1, gC, gS, w, ynew, err, Cn, Sn);
    if (!locating) {
      fCn = Cn;
      fSn = Sn;
    }

    if (locating) {
      loc_it++;
      double Fm[E];
      M::events(t + hs, ynew, p, Fm);
      const int js = jstar;
      double fj = Fm[0];
#pragma unroll
      for (int j = 1; j < E; j++)
        if (j == js) fj = Fm[j];
      double fold = F[0], tolj = pr.evt_tol[0];
#pragma unroll
      for (int j = 1; j < E; j++)
        if (j == js) { fold = F[j]; tolj = pr.evt_tol[j]; }
      if (dabs_le(fj, tolj)) {
        hi = hs;
#pragma unroll
        for (int m = 0; m < n; m++) yhi[m] = ynew[m];
        finish_location(pr);
        return;
      }
      const bool pre = dpos(fj) == dpos(fold);
      // F at the bracket's lower end, kept in theta_a from here on (theta_a
      // itself has been tried; lo is still 0 after a first verification
      // point past the root)
      theta_a = pre ? fj : (loc_phase == 0 ? fold : theta_a);
      if (pre) {
        lo = hs;
      } else {
        hi = hs;
#pragma unroll
        for (int m = 0; m < n; m++) yhi[m] = ynew[m];
      }
      // after theta_a: verify theta_b only if the root lies to its right
      loc_phase = (loc_phase == 0 && pre) ? 1 : 2;
      return;
    }

    steps++;
    if constexpr (SCHEME == kRKCK45) {
      // error ratio and step-size control (Sec. 3, Sec. 6.5)
      // max_m |err_m| / sc_m with a single reciprocal: every ratio is brought
      // over the common denominator prod_m sc_m.  Comparisons, maxima and
      // finiteness tests run on the integer pipe (all operands >= 0).
      double sc[n], num[n];
#pragma unroll
      for (int m = 0; m < n; m++) sc[m] = fma(pr.rtol[m], dmax_nn(dabs(y[m]), dabs(ynew[m])), pr.atol[m]);
      double den = 1.0;
#pragma unroll
      for (int m = 0; m < n; m++) {
        num[m] = dabs(err[m]);
#pragma unroll
        for (int k = 0; k < n; k++)
          if (k != m) num[m] *= sc[k];
        den *= sc[m];
      }
      double nmax = num[0];
#pragma unroll
      for (int m = 1; m < n; m++) nmax = dmax_nn(nmax, num[m]);  // NaN propagates
      double errr = nmax * recip_nr(den);  // den normal and finite here (else below)
      // den below the smallest normal double (the reciprocal flushes it),
      // infinite, or NaN anywhere: one division per ratio, NaN kept
      if (dbits(den) < dbits(2.2250738585072014e-308) || !dfinite(den) || !dfinite(nmax)) {
        errr = 0.0;
#pragma unroll
        for (int m = 0; m < n; m++) {
          const double r = fabs(err[m]) / sc[m];
          errr = (r > errr || isnan(r)) ? r : errr;
        }
      }
      bool finite = dfinite(errr);
#pragma unroll
      for (int m = 0; m < n; m++) finite = finite && dfinite(ynew[m]);
      const bool at_min = dbits(hs) <= dbits(pr.hmin);
      if (!finite) {
        nrej++;
        if (at_min) status = kStHminNaN;
        else h = dmax_nn(pr.shrink * hs, pr.hmin);
        return;
      }
      // new step factor 0.9 err^(-1/5), clamped to [shrink, grow]
      double fac;
      if (dbits(errr) <= dbits(pr.err_grow)) {
        fac = pr.grow;
      } else if (dbits(errr) >= dbits(pr.err_shrink)) {
        fac = pr.shrink;
      } else {
        fac = dclamp_nn(0.9 * rpow_fifth(errr), pr.shrink, pr.grow);
      }
      if (dbits(errr) > dbits(1.0) && !at_min) {
        nrej++;
        h = dclamp_nn(hs * fac, pr.hmin, pr.hmax);
        return;
      }
      hnext = dclamp_nn(hs * fac, pr.hmin, pr.hmax);
    } else {
      bool finite = true;
#pragma unroll
      for (int m = 0; m < n; m++) finite = finite && dfinite(ynew[m]);
      if (!finite) {
        nrej++;
        status = kStHminNaN;
        return;
      }
    }

    const double tnew = last ? t1 : t + hs;
#pragma unroll
    for (int j = 0; j < E; j++) det[j] = false;
    if (pr.events_on) {
      double Fn[E];
      M::events(tnew, ynew, p, Fn);
      int js = -1;
#pragma unroll
      for (int j = 0; j < E; j++) {
        if (!leaving[j] && crossed(pr, j, F[j], Fn[j])) {
          det[j] = true;
          js = j;
        }
      }
      if (js >= 0) {
        double fj = Fn[0], tolj = pr.evt_tol[0];
#pragma unroll
        for (int j = 1; j < E; j++)
          if (j == js) { fj = Fn[j]; tolj = pr.evt_tol[j]; }
        if (!dabs_le(fj, tolj)) {
          // configuration a of Sec. 4: the step jumped over the zone --
          // locate the root in the step size from (t, y), bracketed.  The
          // bracket [0, hs] is first narrowed to theta* +- 1e-6 hs around the
          // root of the cubic Hermite interpolant of F (end values and
          // slopes; one extra right-hand side at the step's end), verified by
          // two trial steps; secant steps, with a bisection every fourth
          // trial, then run inside whatever bracket the verification leaves.
          locating = true;
          jstar = js;
          loc_it = 0;
          lo = 0.0;
          hi = hs;
#pragma unroll
          for (int m = 0; m < n; m++) yhi[m] = ynew[m];
          double fold = F[0];
#pragma unroll
          for (int j = 1; j < E; j++)
            if (j == js) fold = F[j];
          const double theta =
              predict_root(js, t, hs, fold, fj, M::event_rate(js, k1), ynew[0], n > 1 ? ynew[1] : 0.0,
                           n > 2 ? ynew[2] : 0.0, n > 3 ? ynew[3] : 0.0, a.p + sys, (long long)a.ld,
                           a.pr.mc[0], a.pr.mc[1], a.pr.mc[2], Cn, Sn, w);
          const double delta = 1e-6 * hs;
          theta_a = theta - delta;
          theta_b = theta + delta;
          loc_phase = (theta == theta) ? 0 : 2;  // NaN: refine the whole step
          if (loc_phase == 2) theta_a = fold;      // F at lo = 0
          return;
        }
      }
    }
    accept(pr, tnew, ynew, last, false);
  }
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Per-sweep launch with spt systems per thread: the system after `sys` for
// this thread (sys + G with G threads in the grid, at most spt per thread),
// or N when there is none.  Out of line: it runs once per system and keeps
// its registers out of the step loop.
static __device__ __noinline__ int next_static_system(int sys, int N, int spt) {
  const long long G = (long long)gridDim.x * blockDim.x;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nx = (long long)sys + G;
  return (nx < N && nx < g + (long long)spt * G) ? (int)nx : N;
}

// Launch bounds of the integrator kernels: at most M::kMaxThreads per block
// and at least M::kMinBlocks resident blocks of that size per SM, which caps
// the registers per thread at 65536 / (kMaxThreads x kMinBlocks) (more
// resident warps keep the FP64 pipe fed).  Both can be overridden at build
// time (ODEGPU_MAX_THREADS, ODEGPU_MIN_BLOCKS for all models).
#ifdef ODEGPU_MAX_THREADS
#define ODEGPU_MAX_THREADS_OF(M) ODEGPU_MAX_THREADS
#else
#define ODEGPU_MAX_THREADS_OF(M) M::kMaxThreads
#endif
#ifdef ODEGPU_MIN_BLOCKS
#define ODEGPU_MIN_BLOCKS_OF(M) ODEGPU_MIN_BLOCKS
#else
#define ODEGPU_MIN_BLOCKS_OF(M) M::kMinBlocks
#endif

// ---- the kernel --------------------------------------------------------------
template <class M, int SCHEME, int PREC, bool PERSIST>
__global__ void __launch_bounds__(ODEGPU_MAX_THREADS_OF(M), ODEGPU_MIN_BLOCKS_OF(M)) ode_kernel(const KArgs a) {
  using L_t = Lane<M, SCHEME, PREC>;
  using T = typename L_t::T;
  L_t L;
#pragma unroll
  for (int m = 0; m < 3; m++) L.mct[m] = (T)a.pr.mc[m];
  {
    double mcd[3] = {a.pr.mc[0], a.pr.mc[1], a.pr.mc[2]};
    L.w = M::omega(mcd);
  }
  L.tab = nullptr;
  L.tab_n = 0;
  L.tab_t0 = L.tab_t1 = 0.0;
  L.use_tab = false;
  if constexpr (SCHEME == kRK4 && Stepper<M, SCHEME, PREC>::kRotate) {
    // Fixed-step RK4 on a shared time grid (the paper's iterated Solve over
    // forcing periods, Sec. 7.1.1): the forcing at every stage time of the
    // slice is the same for all systems whose slice has the same (t0, t1), so
    // the block tabulates (cos, sin)(omega t) at the stage times of one slice
    // once: that of its first system (per-sweep form) or of system 0
    // (persistent form, whose systems are not known in advance).  Thread 0 walks the step sequence exactly as a lane
    // does (t accumulates t + h; the last step is clipped to t1), writing the
    // times t_i (entry 2 i), t_i + h / 2 (2 i + 1) and the end t_i + h of the
    // last step (2 n); then the block evaluates them.  Systems on that grid
    // read the table for their first tab_n steps; others (a different time
    // domain, another slice in a moving time domain) rotate their own anchor.
    extern __shared__ double2 s_tab[];
    if (a.tab_cap > 0) {
      __shared__ double s_t0, s_t1;
      __shared__ int s_n;
      if (threadIdx.x == 0) {
        const long long first = PERSIST ? 0 : (long long)blockIdx.x * blockDim.x;
        const int s0 = (int)(first < a.N ? first : a.N - 1);
        const double t0 = a.td[s0], t1 = a.td[(size_t)a.ld + s0];
        double nst = ceil((t1 - t0) / a.h0 - 1e-9);
        nst = nst < 1.0 ? 1.0 : nst;
        const double h = (t1 - t0) / nst;
        int ns = 0;
        bool reached = false;  // the walk ended with the clipped last step
        if (t0 < t1 && 2.0 * nst + 1.0 <= (double)a.tab_cap) {
          double t = t0;
          for (; 2 * ns + 2 < a.tab_cap; ns++) {  // writes entries 2 ns .. 2 ns + 2 < tab_cap
            s_tab[2 * ns].x = t;
            if (t1 - t <= h * (1.0 + 1e-9)) {
              const double hs = t1 - t;
              s_tab[2 * ns + 1].x = t + 0.5 * hs;
              s_tab[2 * ns + 2].x = t + hs;
              ns++;
              reached = true;
              break;
            }
            s_tab[2 * ns + 1].x = t + 0.5 * h;
            t = t + h;
          }
        }
        if (!reached) ns = 0;
        s_t0 = t0;
        s_t1 = t1;
        s_n = ns;
      }
      __syncthreads();
      const int ns = s_n;
      for (int j = threadIdx.x; j <= 2 * ns && ns > 0; j += blockDim.x) {
        double sj, cj;
        sincos(L.w * s_tab[j].x, &sj, &cj);
        s_tab[j] = make_double2(cj, sj);
      }
      __syncthreads();
      if (ns > 0) {
        L.tab = s_tab;
        L.tab_n = ns;
        L.tab_t0 = s_t0;
        L.tab_t1 = s_t1;
      }
    }
  }

  // Persistent form.  Thread i of the grid starts with system i, as in the
  // per-sweep grid: the hardware spreads consecutive blocks over the SMs, so
  // every SM starts with an even sample of the parameter grid (a queue-first
  // start hands each SM the systems its warps happen to pop first, a random
  // sample whose cost can differ by tens of percent between SMs when no
  // refill follows).  The G = gridDim.x * blockDim.x systems after them are
  // handed out by the device queue as lanes free up, in one of two orders
  // (the autotuner tries both):
  //  mode 1: warp-aggregated pops -- the lanes that ask together take
  //    consecutive slots, and slot 32 c + r holds system G + 32 ((c *
  //    queue_stride) mod chunks) + r.  So a warp works on neighbouring
  //    systems of the parameter grid (similar step counts: the "clustering"
  //    of Sec. 7.2), while chunks popped one after another lie far apart in
  //    the grid, which balances cheap and expensive regions across SMs;
  //  mode 2: every lane pops the next system in index order on its own (the
  //    lanes of a warp hold systems in the order they freed up).
  const unsigned int G = gridDim.x * blockDim.x;
  const unsigned int nq = (unsigned int)a.N > G ? (unsigned int)a.N - G : 0u;
  const unsigned int chunks = (nq + 31u) / 32u;
  auto pop = [&]() -> int {
    namespace cg = cooperative_groups;
    if (a.queue_mode == 2) {
      const unsigned int x = atomicAdd(a.queue_head, 1u);
      return x < nq ? (int)(G + x) : a.N;
    }
    for (;;) {
      const cg::coalesced_group g = cg::coalesced_threads();
      unsigned int base = 0;
      if (g.thread_rank() == 0) base = atomicAdd(a.queue_head, g.size());
      base = g.shfl(base, 0);
      const unsigned int q = base + g.thread_rank();
      const unsigned int c = q >> 5;
      if (c >= chunks) return a.N;  // queue exhausted
      const unsigned int pc = (unsigned int)(((unsigned long long)c * a.queue_stride) % chunks);
      const unsigned int sys = G + pc * 32u + (q & 31u);
      if (sys < (unsigned int)a.N) return (int)sys;  // else: the unused tail of the last chunk
    }
  };
  bool active;
  // per-sweep form with several systems per thread: the k-th system of thread
  // g is g + k G (G threads in the grid), so a warp always holds neighbours;
  // k follows from the system index, so no register carries it
  L.sys = blockIdx.x * blockDim.x + threadIdx.x;
  active = L.sys < a.N;
  bool fresh = active;  // a new system is loaded and its slice must begin

  // Resolve slice / system ends (also zero-length slices) until the lane has
  // a slice to integrate or no work at all.
  auto next_system = [&]() {
    if constexpr (PERSIST) {
      L.sys = pop();
      active = L.sys < a.N;
      fresh = active;
    } else {
      active = false;
      if (a.spt > 1) {
        L.sys = next_static_system(L.sys, a.N, a.spt);
        active = L.sys < a.N;
        fresh = active;
      }
    }
  };
  auto settle = [&]() {
    while (active) {
      if (fresh) {
        fresh = false;
        if (!L.load(a)) {  // nothing to run for this slot in this launch
          next_system();
          continue;
        }
        L.begin_slice(a);
      }
      if (L.status == kStNone) return;
      L.end_slice(a);
      if (L.slice < L.my_slices) {
        L.begin_slice(a);
        continue;
      }
      L.store(a);
      next_system();
    }
  };

  // Watchdog: a thread that has run longer than time_limit_ns stops its
  // system with kStTimeout, raises flags[0] and takes no further work, so no
  // launch can run unbounded (e.g. a system crawling at the minimum step).
  //
  // Warp-synchronous slices (a.warp_sync): a lane whose slice has ended waits
  // until every lane of its warp has ended its slice, and then they all
  // start the next one together.  Lanes of a warp drift apart by their
  // different step counts; re-aligning them at every slice keeps their
  // steps, event locations and slice starts (which evaluate the forcing
  // anchor) in step with each other, at the price of waiting for the
  // warp's slowest lane in every slice.  Results do not depend on it.
  const unsigned long long t_start = globaltimer_ns();
  unsigned int wd = 0;
  bool at_boundary = false;
  settle();
  while (__any_sync(0xffffffffu, active)) {
    if (active && !at_boundary) {
      L.trial(a);
      if (L.status != kStNone) {
        if (a.warp_sync) at_boundary = true;
        else settle();
      }
      if (active && a.time_limit_ns > 0 && ((++wd & 1023u) == 0u) &&
          globaltimer_ns() - t_start > (unsigned long long)a.time_limit_ns) {
        L.status = kStTimeout;
        L.store(a);
        atomicExch(a.flags, 1);
        active = false;
        at_boundary = false;
      }
    }
    if (a.warp_sync && __all_sync(0xffffffffu, !active || at_boundary)) {
      if (active) {
        at_boundary = false;
        settle();
      }
    }
  }
}

}  // namespace odegpu

#include "serve.cuh"

namespace odegpu {

// Kernel lookup for one model: every (scheme, precision, launch form) variant;
// launch form 3 is the resident serving kernel.
template <class M>
const void* lookup_kernel(int scheme, int prec, int persistent) {
  if (persistent == 3) return lookup_serve_kernel<M>(scheme, prec);
  if (prec == kFP64) {
    if (scheme == kRK4)
      return persistent ? (const void*)ode_kernel<M, kRK4, kFP64, true>
                        : (const void*)ode_kernel<M, kRK4, kFP64, false>;
    return persistent ? (const void*)ode_kernel<M, kRKCK45, kFP64, true>
                      : (const void*)ode_kernel<M, kRKCK45, kFP64, false>;
  }
  if constexpr (M::kHasFP32) {
    if (scheme == kRK4)
      return persistent ? (const void*)ode_kernel<M, kRK4, kFP32RHS, true>
                        : (const void*)ode_kernel<M, kRK4, kFP32RHS, false>;
    return persistent ? (const void*)ode_kernel<M, kRKCK45, kFP32RHS, true>
                      : (const void*)ode_kernel<M, kRKCK45, kFP32RHS, false>;
  }
  return nullptr;
}

}  // namespace odegpu
