// models.cuh -- the pre-declared device hooks of the paper (Sec. 6.5-6.8) for
// each compiled model: right-hand side, event functions, event action,
// accessories and initialization.  They are inlined into the integrator
// kernels of the same translation unit (Sec. 6.9: hooks compiled in a
// separate module cost about 14% on the paper's hardware).
//
// Template parameter T of rhs() is the stage precision: double, or float for
// the FP32 right-hand-side form.
#pragma once

#include <math_constants.h>

#include "bits.cuh"
#include "common.cuh"

namespace odegpu {

__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }

// Time dependence seen by a right-hand-side evaluation: the stage time t and,
// for harmonically forced models, c = cos(omega t) and s = sin(omega t) of
// the model's forcing frequency omega (supplied by the integrator, which
// advances them by angle addition instead of calling cos per stage).
template <class T>
struct Stage {
  T t;
  T c;
  T s;
};

enum Forcing { kNoForcing = 0, kCosForcing = 1, kSinCosForcing = 2 };

// x^(-1/5) for x > 0: binary32 seed refined by two binary64 Newton steps for
// z^-5 = x (z <- z + z (1 - x z^5) / 5; the error goes ~2e-7 -> ~1e-13 ->
// rounding).
__device__ __forceinline__ double rfifth_root(double x) {
  double z = (double)exp2f(-0.2f * __log2f((float)x));
#pragma unroll
  for (int it = 0; it < 2; it++) {
    const double z2 = z * z;
    z = fma(0.2 * z, fma(-x, z2 * z2 * z, 1.0), z);
  }
  return z;
}

// 1 / x for finite, normal x: the hardware's approximate reciprocal
// (rcp.approx.ftz.f64, about 2^-23 relative) refined by two Newton-Raphson
// steps r <- r + r (1 - x r), each of which squares the relative error, to
// within an ulp or two -- four FMAs instead of a correctly rounded division.
__device__ __forceinline__ double recip_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}

// rx^e with rx = 1 / x for the polytropic exponent e = 3 gamma.  When 5 e is a
// small integer k (gamma = 1, 1.4 or 5/3 give k = 15, 21, 25) this is
// rx^(k div 5) * (x^(-1/5))^(k mod 5): a few multiplications and one
// Newton-refined fifth root instead of a general pow().  Other exponents,
// and arguments outside the binary32 seed's range, take pow().
__device__ __forceinline__ double polytropic_pow(double x, double rx, double e) {
  // 5 e within rounding of an integer (3 * 1.4 is 4.1999999999999993 in
  // binary64): the exponent is then taken as that integer over 5.  The
  // nearest integer comes from the 1.5 * 2^52 shifter (its low word holds it)
  // and the range tests compare bit patterns on the integer pipe, so the
  // test costs four binary64 operations per call.
  constexpr double kShift = 6755399441055744.0;  // 1.5 * 2^52
  const double k5 = 5.0 * e;
  const double ks = k5 + kShift;
  const int k = __double2loint(ks);
  const bool near_int = dabs_le(k5 - (ks - kShift), 1e-12 * k5);
  if (near_int && k >= 0 && k <= 60 && dgt(x, 1e-30) && dlt(x, 1e30)) {
    const int q = k / 5, r = k % 5;
    // rx^q by repeated squaring (q <= 12)
    double v = 1.0, b = rx;
#pragma unroll
    for (int bit = 0; bit < 4; bit++) {
      if (q & (1 << bit)) v *= b;
      if (bit < 3) b *= b;
    }
    if (r) {
      const double f = rfifth_root(x);
      double fr = f;
      for (int i = 1; i < r; i++) fr *= f;
      v *= fr;
    }
    return v;
  }
  return pow(rx, e);
}

// Ordinary accessories shared by all models (Sec. 6.7): running maximum and
// minimum of y1 over accepted points, with their times.
__device__ __forceinline__ void acc_minmax(double t, double y1, double* a) {
  // compared on the integer pipe (finite values; bits.cuh)
  if (dgt(y1, a[0])) { a[0] = y1; a[1] = t; }
  if (dlt(y1, a[2])) { a[2] = y1; a[3] = t; }
}

// --------------------------------------------------------------------------
// Duffing oscillator, Eqs. (1)-(2):
//   y1' = y2,  y2' = delta y1 - c3 y1^3 - k y2 + B cos(omega t)
// p = (k, B); model constants mc = (delta, c3, omega).
// Event 0: F = y2 (extrema of y1).  Accessories a0..a3 min/max, a4/a5 the
// first detected event-0 point, a6 its detection count.
// --------------------------------------------------------------------------
struct Duffing {
  static constexpr int N = 2, P = 2, A = 7, E = 1;
  static constexpr bool kHasFP32 = true;
  static constexpr int kMinBlocks = 2;  // launch bound (registers per thread)
  static constexpr int kMaxThreads = 256;
  static constexpr int kForcing = kCosForcing;  // cos(omega t), omega = mc[2]
  static constexpr bool kUnitPeriodForcing = false;

  template <class T>
  static __device__ __forceinline__ T omega(const T (&mc)[3]) { return mc[2]; }
  template <class T>
  static __device__ __forceinline__ void rhs(const Stage<T>& st, const T (&y)[N], const T (&p)[P],
                                             const T (&mc)[3], T (&f)[N]) {
    f[0] = y[1];
    // delta y1 - c3 y1^3 - k y2 + B cos(omega t), as y1 (delta - c3 y1^2) ...
    f[1] = y[0] * (mc[0] - mc[1] * (y[0] * y[0])) - p[0] * y[1] + p[1] * st.c;
  }
  static __device__ __forceinline__ void events(double, const double (&y)[N], const double (&)[P],
                                                double (&F)[E]) {
    F[0] = y[1];
  }
  static __device__ __forceinline__ void action(int, double (&)[N], const double (&)[P]) {}
  // dF_j/dt from the right-hand side f (F0 = y2)
  template <class T>
  static __device__ __forceinline__ double event_rate(int, const T (&f)[N]) { return (double)f[1]; }
  static __device__ __forceinline__ void acc_init(double t, const double (&y)[N], double (&a)[A]) {
    a[0] = y[0]; a[1] = t; a[2] = y[0]; a[3] = t; a[4] = y[0]; a[5] = t; a[6] = 0.0;
  }
  static __device__ __forceinline__ void acc_ordinary(double t, const double (&y)[N], double (&a)[A]) {
    acc_minmax(t, y[0], a);
  }
  static __device__ __forceinline__ void acc_event(int j, int cnt, double t, const double (&y)[N],
                                                   double (&a)[A]) {
    if (j == 0) {
      a[6] = (double)cnt;
      if (cnt == 1) { a[4] = y[0]; a[5] = t; }
    }
  }  // Finalization hook (Sec. 6.8) on the state and accessories: nothing to do
  static __device__ __forceinline__ void finalize(double (&)[N], double (&)[A]) {}
};

// --------------------------------------------------------------------------
// Keller-Miksis bubble, dimensionless form Eqs. (12)-(15) with the
// coefficients C0..C12 of Eqs. (16)-(28) as per-system parameters; t is the
// dimensionless time tau (periods of the first excitation).
// Event 0: F = y2.  Accessories a0..a3 min/max of y1 with times.
// --------------------------------------------------------------------------
struct KellerMiksis {
  static constexpr int N = 2, P = 13, A = 4, E = 1;
  static constexpr bool kHasFP32 = false;
  static constexpr int kMinBlocks = 1;  // launch bound (registers per thread)
  // 65536 / 384 = 170 registers: six 64-thread blocks per SM, no spills
  static constexpr int kMaxThreads = 384;
  static constexpr int kForcing = kSinCosForcing;  // sin, cos of 2 pi tau
  static constexpr bool kUnitPeriodForcing = true;  // omega = 2 pi

  template <class T>
  static __device__ __forceinline__ T omega(const T (&)[3]) { return (T)(2.0 * CUDART_PI); }
  template <class T>
  static __device__ __forceinline__ void rhs(const Stage<T>& st, const T (&y)[N], const T (&C)[P],
                                             const T (&)[3], T (&f)[N]) {
    const double y1 = y[0], y2 = y[1];
    // both reciprocals (1 / y1 and 1 / den) from one: r = 1 / (y1 den)
    const double den = y1 - C[9] * y1 * y2 + C[4] * C[9];
    const double r = recip_nr(y1 * den);
    const double rx = den * r;
    const double s1 = st.s, c1 = st.c;  // sin, cos of 2 pi tau
    double s2 = 0.0, c2 = 0.0;
    // second drive sin(2 pi C11 tau + theta): sincospi reduces its argument
    // exactly (theta / pi is rounded once; theta = 0 in the paper's scans)
    if (C[6] != 0.0 || C[8] != 0.0) sincospi(fma(2.0 * C[11], st.t, C[12] * (1.0 / CUDART_PI)), &s2, &c2);
    const double one_c9y2 = 1.0 + C[9] * y2;
    const double num = (C[0] + C[1] * y2) * polytropic_pow(y1, rx, C[10]) - C[2] * one_c9y2 - C[3] * rx -
                       C[4] * y2 * rx - (1.0 - C[9] * y2 * (1.0 / 3.0)) * 1.5 * y2 * y2 -
                       (C[5] * s1 + C[6] * s2) * one_c9y2 - y1 * (C[7] * c1 + C[8] * c2);
    f[0] = y2;
    f[1] = num * (y1 * r);
  }
  static __device__ __forceinline__ void events(double, const double (&y)[N], const double (&)[P],
                                                double (&F)[E]) {
    F[0] = y[1];
  }
  static __device__ __forceinline__ void action(int, double (&)[N], const double (&)[P]) {}
  template <class T>
  static __device__ __forceinline__ double event_rate(int, const T (&f)[N]) { return (double)f[1]; }
  static __device__ __forceinline__ void acc_init(double t, const double (&y)[N], double (&a)[A]) {
    a[0] = y[0]; a[1] = t; a[2] = y[0]; a[3] = t;
  }
  static __device__ __forceinline__ void acc_ordinary(double t, const double (&y)[N], double (&a)[A]) {
    acc_minmax(t, y[0], a);
  }
  static __device__ __forceinline__ void acc_event(int, int, double, const double (&)[N], double (&)[A]) {}  // Finalization hook (Sec. 6.8) on the state and accessories: nothing to do
  static __device__ __forceinline__ void finalize(double (&)[N], double (&)[A]) {}
};

// --------------------------------------------------------------------------
// Pressure relief valve, Eqs. (29)-(31), impact law Eqs. (32)-(34);
// p = (kappa, delta, beta, q, r).  Event 0: F = y2 (maxima of the
// displacement, the Poincare section of Sec. 7.3); event 1: F = y1 (contact
// with the seat), whose action is y2 <- -r y2.  Accessories a0..a3 min/max
// of y1 with times, a4 the number of impacts.
// --------------------------------------------------------------------------
struct Valve {
  static constexpr int N = 3, P = 5, A = 5, E = 2;
  static constexpr bool kHasFP32 = true;
  static constexpr int kMinBlocks = 2;  // launch bound (registers per thread)
  static constexpr int kMaxThreads = 256;
  static constexpr int kForcing = kNoForcing;
  static constexpr bool kUnitPeriodForcing = false;

  template <class T>
  static __device__ __forceinline__ T omega(const T (&)[3]) { return (T)0; }
  template <class T>
  static __device__ __forceinline__ void rhs(const Stage<T>&, const T (&y)[N], const T (&p)[P],
                                             const T (&)[3], T (&f)[N]) {
    f[0] = y[1];
    f[1] = -p[0] * y[1] - (y[0] + p[1]) + y[2];
    f[2] = p[2] * (p[3] - y[0] * sqrt_t(y[2]));
  }
  static __device__ __forceinline__ void events(double, const double (&y)[N], const double (&)[P],
                                                double (&F)[E]) {
    F[0] = y[1];
    F[1] = y[0];
  }
  static __device__ __forceinline__ void action(int j, double (&y)[N], const double (&p)[P]) {
    if (j == 1) y[1] = -p[4] * y[1];
  }
  // F0 = y2, F1 = y1
  template <class T>
  static __device__ __forceinline__ double event_rate(int j, const T (&f)[N]) {
    return j == 0 ? (double)f[1] : (double)f[0];
  }
  static __device__ __forceinline__ void acc_init(double t, const double (&y)[N], double (&a)[A]) {
    a[0] = y[0]; a[1] = t; a[2] = y[0]; a[3] = t; a[4] = 0.0;
  }
  static __device__ __forceinline__ void acc_ordinary(double t, const double (&y)[N], double (&a)[A]) {
    acc_minmax(t, y[0], a);
  }
  static __device__ __forceinline__ void acc_event(int j, int cnt, double, const double (&)[N],
                                                   double (&a)[A]) {
    if (j == 1) a[4] = (double)cnt;
  }  // Finalization hook (Sec. 6.8) on the state and accessories: nothing to do
  static __device__ __forceinline__ void finalize(double (&)[N], double (&)[A]) {}
};

// --------------------------------------------------------------------------
// Bouncing ball: y1' = y2, y2' = -g, p = (g, r); event 0: F = y1 with the
// impact y2 <- -r y2.  Accessories a0..a3 min/max with times, a4 the time of
// the last impact, a5 the velocity just before it.
// --------------------------------------------------------------------------
struct Bounce {
  static constexpr int N = 2, P = 2, A = 6, E = 1;
  static constexpr bool kHasFP32 = true;
  static constexpr int kMinBlocks = 2;  // launch bound (registers per thread)
  static constexpr int kMaxThreads = 256;
  static constexpr int kForcing = kNoForcing;
  static constexpr bool kUnitPeriodForcing = false;

  template <class T>
  static __device__ __forceinline__ T omega(const T (&)[3]) { return (T)0; }
  template <class T>
  static __device__ __forceinline__ void rhs(const Stage<T>&, const T (&y)[N], const T (&p)[P],
                                             const T (&)[3], T (&f)[N]) {
    f[0] = y[1];
    f[1] = -p[0];
  }
  static __device__ __forceinline__ void events(double, const double (&y)[N], const double (&)[P],
                                                double (&F)[E]) {
    F[0] = y[0];
  }
  static __device__ __forceinline__ void action(int j, double (&y)[N], const double (&p)[P]) {
    if (j == 0) y[1] = -p[1] * y[1];
  }
  // F0 = y1
  template <class T>
  static __device__ __forceinline__ double event_rate(int, const T (&f)[N]) { return (double)f[0]; }
  static __device__ __forceinline__ void acc_init(double t, const double (&y)[N], double (&a)[A]) {
    a[0] = y[0]; a[1] = t; a[2] = y[0]; a[3] = t; a[4] = t; a[5] = y[1];
  }
  static __device__ __forceinline__ void acc_ordinary(double t, const double (&y)[N], double (&a)[A]) {
    acc_minmax(t, y[0], a);
  }
  static __device__ __forceinline__ void acc_event(int j, int, double t, const double (&y)[N],
                                                   double (&a)[A]) {
    if (j == 0) { a[4] = t; a[5] = y[1]; }
  }  // Finalization hook (Sec. 6.8) on the state and accessories: nothing to do
  static __device__ __forceinline__ void finalize(double (&)[N], double (&)[A]) {}
};


// --------------------------------------------------------------------------
// Duffing with its linearisation attached in polar coordinates for the
// largest Lyapunov exponent, Eqs. (3)-(6): y3 is the radius and y4 the angle
// of a tangent vector of (y1, y2),
//   y3' = y3 ((1 + g1) sin y4 cos y4 + g2 sin^2 y4),
//   y4' = -sin^2 y4 + (g1 cos y4 + g2 sin y4) cos y4,
// g1 = dF2/dy1 = delta - 3 c3 y1^2, g2 = dF2/dy2 = -k.  p and mc as Duffing.
// Event 0: F = y2.  Accessories a0..a3 min/max of y1 with times; a4 = ln y3
// at the slice end, where the Finalization hook restarts the radius from one
// (Eq. (7): the exponent is the mean of ln y3(t_n) per unit time) and reduces
// the angle modulo 2 pi.
// --------------------------------------------------------------------------
struct DuffingLyapunov {
  static constexpr int N = 4, P = 2, A = 5, E = 1;
  static constexpr bool kHasFP32 = false;
  static constexpr int kMinBlocks = 1;  // launch bound (registers per thread)
  static constexpr int kMaxThreads = 256;
  static constexpr int kForcing = kCosForcing;  // cos(omega t), omega = mc[2]
  static constexpr bool kUnitPeriodForcing = false;

  template <class T>
  static __device__ __forceinline__ T omega(const T (&mc)[3]) { return mc[2]; }
  template <class T>
  static __device__ __forceinline__ void rhs(const Stage<T>& st, const T (&y)[N], const T (&p)[P],
                                             const T (&mc)[3], T (&f)[N]) {
    const T y1s = y[0] * y[0];
    f[0] = y[1];
    f[1] = y[0] * (mc[0] - mc[1] * y1s) - p[0] * y[1] + p[1] * st.c;
    const T g1 = mc[0] - (T)3 * mc[1] * y1s;
    T s, c;
    sincos_t(y[3], &s, &c);
    const T ss = s * s;
    f[2] = y[2] * (((T)1 + g1) * (s * c) - p[0] * ss);
    f[3] = (g1 * c - p[0] * s) * c - ss;
  }
  static __device__ __forceinline__ void events(double, const double (&y)[N], const double (&)[P],
                                                double (&F)[E]) {
    F[0] = y[1];
  }
  static __device__ __forceinline__ void action(int, double (&)[N], const double (&)[P]) {}
  template <class T>
  static __device__ __forceinline__ double event_rate(int, const T (&f)[N]) { return (double)f[1]; }
  static __device__ __forceinline__ void acc_init(double t, const double (&y)[N], double (&a)[A]) {
    a[0] = y[0]; a[1] = t; a[2] = y[0]; a[3] = t; a[4] = 0.0;
  }
  static __device__ __forceinline__ void acc_ordinary(double t, const double (&y)[N], double (&a)[A]) {
    acc_minmax(t, y[0], a);
  }
  static __device__ __forceinline__ void acc_event(int, int, double, const double (&)[N], double (&)[A]) {}
  // Finalization hook (Sec. 6.8): keep the slice's stretch, restart the
  // radius, and bring the angle back to [-pi, pi] (the right-hand side sees
  // it only through sin and cos; an unbounded angle would loosen its
  // relative tolerance)
  static __device__ __forceinline__ void finalize(double (&y)[N], double (&a)[A]) {
    a[4] = log(y[2]);
    y[2] = 1.0;
    y[3] = remainder(y[3], 2.0 * CUDART_PI);
  }
};

}  // namespace odegpu
