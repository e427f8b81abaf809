// fx128.cuh -- 128-bit fixed-point numbers for the exact row sums of the
// power series (Sec. 4.3.2) on the integer pipes.
//
// GB300 retires about two FP64 lanes per clock per SM against 64 or more
// integer lanes, so a sweep whose FP64 adds run one row per lane is bound by
// the FP64 pipe.  A value x is held here as the integer round(x * 2^F) in a
// signed 128-bit word, for a binary point F chosen per component: sums of
// such words are exact (integer adds with carry), so a row's in-edge sum has
// no rounding at all, whatever its length or order; only the conversions
// round (to the nearest multiple of 2^-F on the way in, to the nearest
// double on the way out).
#pragma once

#include <stdint.h>

namespace prgb {

typedef __int128 fx128;
typedef unsigned __int128 ufx128;

// Binary point for a component whose weights sum (L1) to wsum: every value
// the series forms is at most 2^17 * wsum in magnitude (terms and partial
// sums of a cold start are at most wsum / (1 - c); a warm start's guess is
// at most (1 + e^9) wsum, its residual about twice that), so
// F = 110 - (exponent of wsum) leaves them below 2^127.
// The quantum is then 2^-110 wsum.  Clamped so that every conversion below
// stays in the normal double range.
__device__ __forceinline__ int fx_point(double wsum) {
  if (!(wsum > 0.0)) return 0;
  const long long b = __double_as_longlong(wsum);
  const int e = (int)((b >> 52) & 0x7ff) - 1022;  // wsum < 2^e
  const int f = 110 - e;
  return f < -890 ? -890 : (f > 1000 ? 1000 : f);
}

// round(x * 2^F) (half away from zero); |x| * 2^F is below 2^127 by the
// choice of F (a larger value saturates at 2^126 rather than wrapping)
__device__ __forceinline__ fx128 to_fx(double x, int F) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  unsigned long long m = b & 0xfffffffffffffULL;
  if (e) m |= 1ULL << 52;
  const int sh = (e ? e : 1) - 1075 + F;  // x = m * 2^(sh - F)
  ufx128 v;
  if (sh > 74) {
    v = (ufx128)1 << 126;
  } else if (sh >= 0) {
    v = (ufx128)m << sh;
  } else if (sh > -64) {
    v = (ufx128)((m + (1ULL << (-sh - 1))) >> (-sh));
  } else {
    v = 0;
  }
  return (b >> 63) ? -(fx128)v : (fx128)v;
}

// v * 2^-F rounded to the nearest double (ties to even), with integer
// operations only
__device__ __forceinline__ double from_fx(fx128 v, int F) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? 1ULL : 0ULL;
  const ufx128 a = sign ? (ufx128)(-v) : (ufx128)v;
  const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  const ufx128 nrm = a << lz;  // leading one at bit 127
  const unsigned long long top = (unsigned long long)(nrm >> 64), bot = (unsigned long long)nrm;
  unsigned long long mant = top >> 11;  // 53 bits, leading one at bit 52
  const unsigned long long rbit = (top >> 10) & 1ULL;
  const bool sticky = (top & 0x3ffULL) != 0 || bot != 0;
  int ex = (127 - lz) - F;  // value = 1.xxx * 2^ex
  if (rbit && (sticky || (mant & 1ULL))) {
    mant++;
    if (mant >> 53) {
      mant >>= 1;
      ex++;
    }
  }
  const unsigned long long bits =
      (sign << 63) | ((unsigned long long)(ex + 1023) << 52) | (mant & 0xfffffffffffffULL);
  return __longlong_as_double((long long)bits);
}

// A positive double below 1 (c/outdeg) as M 2^-sh with M normalised to
// 64 bits (top bit set), so sh >= 64; zero gives M = 0.
struct FxMul {
  unsigned long long M;
  int sh;
};
__device__ __forceinline__ FxMul fx_mul_of(double x) {
  FxMul r{0ULL, 64};
  if (!(x > 0.0)) return r;
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7ff);
  unsigned long long m = b & 0xfffffffffffffULL;
  if (e) m |= 1ULL << 52;
  else e = 1;
  const int lz = __clzll((long long)m);
  r.M = m << lz;
  r.sh = 1075 - e + lz;  // x = m 2^(e - 1075) = M 2^-(1075 - e + lz)
  return r;
}

// round(v M 2^-sh) (half away from zero), the exact product of a
// fixed-point value and the double that f describes, rounded once: 64-bit
// multiplies on the integer pipes, no floating point.  |result| < |v|.
__device__ __forceinline__ fx128 fx_scale(fx128 v, FxMul f) {
  const bool neg = v < 0;
  const ufx128 a = neg ? (ufx128)(-v) : (ufx128)v;  // below 2^127
  const ufx128 t0 = (ufx128)(unsigned long long)a * f.M;
  const ufx128 t1 = (ufx128)(unsigned long long)(a >> 64) * f.M;  // below 2^127
  // the product is hi 2^64 + w0
  const ufx128 mid = (t0 >> 64) + (ufx128)(unsigned long long)t1;
  const ufx128 hi = ((t1 >> 64) << 64) + mid;
  const unsigned long long w0 = (unsigned long long)t0;
  const int r = f.sh - 64;
  ufx128 q;
  if (r == 0) {
    q = hi + (w0 >> 63);
  } else if (r <= 127) {
    const ufx128 h = hi >> (r - 1);  // the rounding bit is h's lowest
    q = (h >> 1) + (h & 1);
  } else {
    q = 0;
  }
  return neg ? -(fx128)q : (fx128)q;
}

// |v| 2^-F as a float, rounded toward zero (relative error below 2^-23);
// magnitudes under the normal float range give 0.  Integer operations only.
__device__ __forceinline__ float fx_abs_float(fx128 v, int F) {
  if (v == 0) return 0.0f;
  const ufx128 a = v < 0 ? (ufx128)(-v) : (ufx128)v;
  const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  const int e = (127 - lz) - F;  // |v| 2^-F in [2^e, 2^(e+1))
  if (e < -126) return 0.0f;
  if (e > 127) return 3.4028235e38f;
  const unsigned long long top = (unsigned long long)((a << lz) >> 64);  // leading one at bit 63
  const unsigned mant = (unsigned)(top >> 40) & 0x7fffffu;
  return __int_as_float(((e + 127) << 23) | (int)mant);
}

}  // namespace prgb
