// bits.cuh -- binary64 comparisons, minima, maxima and finiteness tests on
// the integer pipe.  On this GPU the binary64 pipe is 1/64 as wide as the
// integer pipe, so the integrator keeps its bookkeeping off it.
//
// The bit patterns of non-negative doubles, read as signed 64-bit integers,
// are ordered like the numbers; dkey() extends that order to both signs
// (flipping the magnitude bits of negative numbers), with -0 just below +0.
// Arguments must not be NaN unless a function says otherwise.
#pragma once

namespace odegpu {

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

__device__ __forceinline__ long long dkey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// x is neither infinite nor NaN
__device__ __forceinline__ bool dfinite(double x) {
  return (dbits(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// |x| <= t for t >= 0 (false for NaN x)
__device__ __forceinline__ bool dabs_le(double x, double t) {
  return (dbits(x) & 0x7fffffffffffffffLL) <= dbits(t);
}

// x > 0 and x < 0 with IEEE semantics for +0 / -0
__device__ __forceinline__ bool dpos(double x) { return dkey(x) > 0; }
__device__ __forceinline__ bool dneg(double x) { return dkey(x) < -1; }

// a <= b, a < b, a > b for any signs (not NaN)
__device__ __forceinline__ bool dle(double a, double b) { return dkey(a) <= dkey(b); }
__device__ __forceinline__ bool dlt(double a, double b) { return dkey(a) < dkey(b); }
__device__ __forceinline__ bool dgt(double a, double b) { return dkey(a) > dkey(b); }

// max / min of non-negative values (a NaN argument yields a NaN result for
// max, which the callers test)
__device__ __forceinline__ double dmax_nn(double a, double b) {
  return __longlong_as_double(max(dbits(a), dbits(b)));
}
__device__ __forceinline__ double dmin_nn(double a, double b) {
  return __longlong_as_double(min(dbits(a), dbits(b)));
}
__device__ __forceinline__ double dabs(double x) {
  return __longlong_as_double(dbits(x) & 0x7fffffffffffffffLL);
}
// clamp of a non-negative value into [lo, hi], 0 <= lo <= hi
__device__ __forceinline__ double dclamp_nn(double x, double lo, double hi) {
  return dmin_nn(dmax_nn(x, lo), hi);
}

}  // namespace odegpu
