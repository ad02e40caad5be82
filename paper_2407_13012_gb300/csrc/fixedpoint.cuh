// Integer fixed-point helpers for the complex128 sweep arithmetic.
//
// The state inside a call is int64 with value = integer * 2^-S; unit-modulus factors
// (phases, mixer diagonals) are Q62 (value = integer * 2^-62).  Every helper uses
// integer instructions only (GB300's float64 pipe retires ~1.75 FMA per SM clock).
// The header compiles for the device and, for the CPU tests, for the host.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define QAOA_HD __host__ __device__ __forceinline__
#else
#define QAOA_HD inline
#endif

namespace qaoa {
namespace fx {

typedef __int128 i128;

QAOA_HD int clz64(unsigned long long a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return a ? __builtin_clzll(a) : 64;
#endif
}

QAOA_HD double bits_to_double(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  union {
    unsigned long long u;
    double d;
  } c;
  c.u = b;
  return c.d;
#endif
}

QAOA_HD unsigned long long double_to_bits(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  union {
    unsigned long long u;
    double d;
  } c;
  c.d = d;
  return c.u;
#endif
}

// round(v / 2^s) for s >= 0, ties toward +infinity
QAOA_HD long long round_shift(i128 v, int s) {
  return s > 0 ? (long long)((v + ((i128)1 << (s - 1))) >> s) : (long long)v;
}

// A value split into 32-bit limbs x = h * 2^32 + l with l signed, |l| <= 2^31 (8-byte
// aligned, so a prepared factor in shared memory loads as three 64-bit words).
struct alignas(8) Limbs {
  int h;
  int l;
};

QAOA_HD Limbs split(long long x) {
  const int l = (int)(unsigned int)(unsigned long long)x;
  const int h = (int)((x - (long long)l) >> 32);
  Limbs r;
  r.h = h;
  r.l = l;
  return r;
}

// a * b + c for 32-bit a, b and a 64-bit c.  On the device this is one multiply-add-wide
// instruction; written as (long long)a * b + c the compiler emits a 64 x 64-bit multiply
// (measured: 8 instead of 3 instructions per product, 74 instead of 42 per complex multiply).
QAOA_HD long long madw(int a, int b, long long c) {
#ifdef __CUDA_ARCH__
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
#else
  return (long long)a * b + c;
#endif
}

// round((a b + c d) / 2^(62 + e)) for a, c with |.| < 2^61 and b, d Q62 with |.| <= 2^62,
// 0 <= e <= 30, from eight 32x32 -> 64-bit products.  x y = xh yh 2^64 + (xh yl + xl yh) 2^32
// + xl yl; the low products enter only through their high words, so the result can differ
// from exact rounding by one unit when the exact value lies within 2^-29 units of a tie.
QAOA_HD long long dot2_q62(Limbs a, Limbs b, Limbs c, Limbs d, int e) {
  const long long P = madw(c.h, d.h, madw(a.h, b.h, 0));
  const long long M = madw(c.l, d.h, madw(c.h, d.l, madw(a.l, b.h, madw(a.h, b.l, 0))));
  const long long Lh = (madw(a.l, b.l, 0) >> 32) + (madw(c.l, d.l, 0) >> 32);
  const long long T = M + Lh;  // value = P 2^64 + T 2^32 (up to the dropped low words)
  if (e <= 2) return (long long)((unsigned long long)P << (2 - e)) + ((T + (1ll << (29 + e))) >> (30 + e));
  return (P + ((T + (1ll << (29 + e))) >> 32)) >> (e - 2);
}

// dot2_q62 without the products of the low limbs: they add at most 2^(1 - e) result units,
// so for e >= 3 the result is within one unit of exact rounding (two fewer 32 x 32-bit
// products per call)
QAOA_HD long long dot2_q62_hi(Limbs a, Limbs b, Limbs c, Limbs d, int e) {
  const long long P = madw(c.h, d.h, madw(a.h, b.h, 0));
  const long long T = madw(c.l, d.h, madw(c.h, d.l, madw(a.l, b.h, madw(a.h, b.l, 0))));
  if (e <= 2) return (long long)((unsigned long long)P << (2 - e)) + ((T + (1ll << (29 + e))) >> (30 + e));
  return (P + ((T + (1ll << (29 + e))) >> 32)) >> (e - 2);
}

// Exact 128-bit products from four 32 x 32-bit limb products each (fused multiply-add-wide
// on the device).  Operands |.| < 2^61: the high limbs are below 2^29 in magnitude, so the
// middle sums stay inside int64; the low-limb difference (two products of magnitude <= 2^62)
// does too.
// a b - c d
QAOA_HD i128 dot2_exact(long long a, long long b, long long c, long long d) {
  const Limbs A = split(a), B = split(b), C = split(c), D = split(d);
  const long long P = madw(-C.h, D.h, madw(A.h, B.h, 0));
  const long long M = madw(A.h, B.l, madw(A.l, B.h, 0)) - madw(C.h, D.l, madw(C.l, D.h, 0));
  const long long L = madw(A.l, B.l, 0) - madw(C.l, D.l, 0);
  return ((i128)P << 64) + ((i128)M << 32) + (i128)L;
}
// a c for a 64-bit a (|a| < 2^62) and a 32-bit c
QAOA_HD i128 mul_wide32(long long a, int c) {
  const Limbs A = split(a);
  return ((i128)madw(A.h, c, 0) << 32) + (i128)madw(A.l, c, 0);
}

// x * u / 2^(62 + e) for complex x (|re|, |im| < 2^61) and a Q62 unit complex u
struct C64 {
  long long x, y;
};

QAOA_HD C64 cmul_q62(long long xr, long long xi, long long ur, long long ui, int e) {
  const Limbs r = split(xr), i = split(xi), ni = split(-xi);
  const Limbs a = split(ur), b = split(ui);
  C64 o;
  o.x = dot2_q62(r, a, ni, b, e);  // xr ur - xi ui
  o.y = dot2_q62(r, b, i, a, e);   // xr ui + xi ur
  return o;
}

// cmul_q62 with dot2_q62_hi (for e >= 3: within one unit of exact rounding)
QAOA_HD C64 cmul_q62_hi(long long xr, long long xi, long long ur, long long ui, int e) {
  const Limbs r = split(xr), i = split(xi), ni = split(-xi);
  const Limbs a = split(ur), b = split(ui);
  C64 o;
  o.x = dot2_q62_hi(r, a, ni, b, e);
  o.y = dot2_q62_hi(r, b, i, a, e);
  return o;
}

// Reference with 128-bit products (one rounding per part); any |x| < 2^63.
QAOA_HD C64 cmul_q62_exact(long long xr, long long xi, long long ur, long long ui, int e) {
  const i128 re = (i128)xr * ur - (i128)xi * ui;
  const i128 im = (i128)xr * ui + (i128)xi * ur;
  C64 o;
  o.x = round_shift(re, 62 + e);
  o.y = round_shift(im, 62 + e);
  return o;
}

// A Q62 unit complex number u = ur + i ui prepared for repeated multiplies: the limbs of ur,
// ui and -ui (the negation done once here instead of once per product).
struct Factor {
  Limbs r, i, ni;
};

QAOA_HD Factor factor(long long ur, long long ui) {
  Factor f;
  f.r = split(ur);
  f.i = split(ui);
  f.ni = split(-ui);
  return f;
}

// x * u / 2^(62 + e) with u given as a Factor (conjugated when CONJ): the real part is
// xr ur + xi (-ui), the imaginary part xr ui + xi ur (for conj(u): xr ur + xi ui and
// xr (-ui) + xi ur).  FULL keeps every limb product (within one unit of exact rounding,
// like cmul_q62); otherwise the low x low products are dropped: within one unit for
// e >= 3 and within three units for e = 0.
template <bool FULL, bool CONJ>
QAOA_HD C64 cmul_factor(long long xr, long long xi, const Factor& f, int e) {
  const Limbs r = split(xr), i = split(xi);
  const Limbs& ui = CONJ ? f.ni : f.i;
  const Limbs& nui = CONJ ? f.i : f.ni;
  C64 o;
  if (FULL) {
    o.x = dot2_q62(r, f.r, i, nui, e);
    o.y = dot2_q62(r, ui, i, f.r, e);
  } else {
    o.x = dot2_q62_hi(r, f.r, i, nui, e);
    o.y = dot2_q62_hi(r, ui, i, f.r, e);
  }
  return o;
}

// float64 of x * 2^-s, correctly rounded (round to nearest, ties to even), assembled from
// the binary64 layout sign | 11-bit biased exponent | 52-bit fraction.  The result must be
// a normal number.
QAOA_HD double to_double(long long x, int s) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = x < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int lz = clz64(a);
  const unsigned long long m = a << lz;  // leading one at bit 63
  unsigned long long keep = m >> 11;     // 53 significant bits
  const unsigned long long rem = m & 0x7FFull;
  keep += (rem > 0x400ull) || (rem == 0x400ull && (keep & 1ull));
  int ex = (63 - lz) - s;
  if (keep >> 53) {
    keep >>= 1;
    ++ex;
  }
  return bits_to_double(sgn | ((unsigned long long)(ex + 1023) << 52) | (keep & ((1ull << 52) - 1)));
}

// float64 of an int128 v * 2^-s (a sticky shift to 62 bits, then to_double)
QAOA_HD double i128_to_double(i128 v, int s) {
  const bool neg = v < 0;
  const unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  long long q;
  int sh = 0;
  if (hi == 0 && (lo >> 62) == 0) {
    q = (long long)lo;
  } else {
    const int nbits = hi ? 128 - clz64(hi) : 64 - clz64(lo);
    sh = nbits - 62;
    const unsigned __int128 mask = (((unsigned __int128)1) << sh) - 1;
    q = (long long)(a >> sh) | ((a & mask) != 0 ? 1 : 0);
  }
  return to_double(neg ? -q : q, s - sh);
}

// round(d * 2^s) as int64 (half away from zero) for |d| 2^s < 2^62
QAOA_HD long long from_double(double d, int s) {
  const unsigned long long bits = double_to_bits(d);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero or subnormal: below every resolution used here
  const long long m = (long long)((bits & ((1ull << 52) - 1)) | (1ull << 52));
  const int sh = ex - 1075 + s;  // value * 2^s = m * 2^sh
  long long r;
  if (sh >= 0) r = sh >= 10 ? (m << 9) : (m << sh);  // clamp; callers stay in range
  else if (sh > -64) r = (m >> (-sh)) + ((m >> (-sh - 1)) & 1);
  else r = 0;
  return (bits >> 63) ? -r : r;
}

// (d mod 1) * 2^64 as an unsigned turn count
QAOA_HD unsigned long long frac_turns(double d) {
  const unsigned long long bits = double_to_bits(d);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return 0ull;
  const unsigned long long m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = ex - 1075 + 64;  // d * 2^64 = m * 2^sh
  unsigned long long t;
  if (sh >= 64) t = 0ull;
  else if (sh >= 0) t = m << sh;  // wraps mod 2^64
  else if (sh > -64) t = (m >> (-sh)) + ((m >> (-sh - 1)) & 1ull);
  else t = 0ull;
  return (bits >> 63) ? (0ull - t) : t;
}

}  // namespace fx
}  // namespace qaoa
