// Host check of the fixed-point helpers in csrc/fixedpoint.cuh against 128-bit exact
// arithmetic and the C library's correctly rounded conversions.  Exit 0 = all good.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>

#include "fixedpoint.cuh"

using namespace qaoa::fx;

static long long q62(double x) { return llrint(ldexp(x, 62)); }

int main() {
  std::mt19937_64 rng(12345);
  int fails = 0;
  long long exact = 0, total = 0;
  std::uniform_real_distribution<double> ang(0.0, 6.283185307179586);
  for (int it = 0; it < 2000000; ++it) {
    const int bits = 1 + (int)(rng() % 61);  // magnitudes from tiny to < 2^61
    const long long lim = (1ll << bits) - 1;
    const long long xr = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
    const long long xi = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
    const double th = ang(rng);
    long long ur = q62(std::cos(th)), ui = q62(std::sin(th));
    if (it % 97 == 0) { ur = 1ll << 62; ui = 0; }
    if (it % 89 == 0) { ur = 0; ui = -(1ll << 62); }
    const int e = (int)(rng() % 14);
    const C64 a = cmul_q62(xr, xi, ur, ui, e);
    const C64 b = cmul_q62_exact(xr, xi, ur, ui, e);
    const long long dx = a.x - b.x, dy = a.y - b.y;
    total += 2;
    exact += (dx == 0) + (dy == 0);
    if (dx > 1 || dx < -1 || dy > 1 || dy < -1) {
      if (fails++ < 5) printf("cmul mismatch x=(%lld,%lld) u=(%lld,%lld) e=%d: %lld %lld vs %lld %lld\n", xr, xi, ur, ui,
                              e, a.x, a.y, b.x, b.y);
    }
  }
  if ((double)exact / (double)total < 0.9999) {
    printf("cmul exact rate too low: %lld / %lld\n", exact, total);
    ++fails;
  }
  // the mixer-diagonal form without low-limb products: within one unit for e >= 3
  for (int it = 0; it < 1000000; ++it) {
    const int bits = 1 + (int)(rng() % 61);
    const long long lim = (1ll << bits) - 1;
    const long long xr = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
    const long long xi = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
    const double th = ang(rng);
    const long long ur = q62(std::cos(th)), ui = q62(std::sin(th));
    const int e = 3 + (int)(rng() % 11);
    const C64 a = cmul_q62_hi(xr, xi, ur, ui, e);
    const C64 b = cmul_q62_exact(xr, xi, ur, ui, e);
    const long long dx = a.x - b.x, dy = a.y - b.y;
    if (dx > 1 || dx < -1 || dy > 1 || dy < -1) {
      if (fails++ < 10) printf("cmul_hi mismatch e=%d: %lld %lld vs %lld %lld\n", e, a.x, a.y, b.x, b.y);
    }
  }
  // prepared factors (and their conjugates): full form within one unit; without the low
  // products within one unit for e >= 3 and within three units for e = 0
  for (int it = 0; it < 1000000; ++it) {
    const int bits = 1 + (int)(rng() % 61);
    const long long lim = (1ll << bits) - 1;
    const long long xr = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
    const long long xi = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
    const double th = ang(rng);
    long long ur = q62(std::cos(th)), ui = q62(std::sin(th));
    if (it % 97 == 0) { ur = 1ll << 62; ui = 0; }
    if (it % 89 == 0) { ur = 0; ui = -(1ll << 62); }
    const Factor f = factor(ur, ui);
    const int e = (it & 1) ? 0 : 3 + (int)(rng() % 11);
    const long long tol_hi = e == 0 ? 3 : 1;
    const C64 b = cmul_q62_exact(xr, xi, ur, ui, e), bc = cmul_q62_exact(xr, xi, ur, -ui, e);
    const C64 a[4] = {cmul_factor<true, false>(xr, xi, f, e), cmul_factor<true, true>(xr, xi, f, e),
                      cmul_factor<false, false>(xr, xi, f, e), cmul_factor<false, true>(xr, xi, f, e)};
    for (int k = 0; k < 4; ++k) {
      const C64& want = (k & 1) ? bc : b;
      const long long tol = k < 2 ? 1 : tol_hi;
      const long long dx = a[k].x - want.x, dy = a[k].y - want.y;
      if (dx > tol || dx < -tol || dy > tol || dy < -tol) {
        if (fails++ < 10) printf("cmul_factor<%d> mismatch e=%d: %lld %lld vs %lld %lld\n", k, e, a[k].x, a[k].y,
                                 want.x, want.y);
      }
    }
  }
  // exact limb products against plain 128-bit arithmetic
  for (int it = 0; it < 1000000; ++it) {
    long long v[4];
    for (int k = 0; k < 4; ++k) {
      const int bits = 1 + (int)(rng() % 60);  // |v| < 2^61
      const long long lim = (1ll << bits) - 1;
      v[k] = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
    }
    if (it % 101 == 0) { v[0] = (1ll << 61) - 1; v[1] = -(1ll << 61) + 1; v[2] = -(1ll << 61) + 1; v[3] = -(1ll << 61) + 1; }
    const __int128 want = (__int128)v[0] * v[1] - (__int128)v[2] * v[3];
    const int c = (int)(unsigned)rng();
    const __int128 want2 = (__int128)v[0] * c;
    if (dot2_exact(v[0], v[1], v[2], v[3]) != want || mul_wide32(v[0], c) != want2) {
      if (fails++ < 10) printf("exact limb product mismatch\n");
    }
  }
  for (int it = 0; it < 1000000; ++it) {
    const long long x = (long long)(rng() >> (rng() % 63)) * ((rng() & 1) ? 1 : -1);
    const int s = (int)(rng() % 120);
    const double ref = ldexp((double)x, -s);  // int64 -> double is correctly rounded
    const double got = to_double(x, s);
    if (x != 0 && got != ref) {
      if (fails++ < 10) printf("to_double(%lld, %d) = %.17g vs %.17g\n", x, s, got, ref);
    }
    const __int128 v = ((__int128)(long long)rng() << (rng() % 60)) + (long long)rng();
    const int s2 = (int)(rng() % 200);
    const double r2 = ldexp((double)v, -s2);
    if (v != 0 && i128_to_double(v, s2) != r2) {
      if (fails++ < 10) printf("i128_to_double mismatch\n");
    }
    const double d = ldexp((double)(long long)(rng() >> 11) - 4503599627370496.0, -(int)(rng() % 60));
    const int s3 = (int)(rng() % 40);
    if (std::fabs(ldexp(d, s3)) < 4.0e18) {
      const long long r3 = llround(ldexp(d, s3));
      if (from_double(d, s3) != r3) {
        if (fails++ < 10) printf("from_double(%.17g, %d) = %lld vs %lld\n", d, s3, from_double(d, s3), r3);
      }
    }
  }
  // frac_turns: fixed points and period 1
  if (frac_turns(0.5) != (1ull << 63) || frac_turns(-0.25) != 3ull << 62 || frac_turns(7.0) != 0ull ||
      frac_turns(0.125) != (1ull << 61)) {
    printf("frac_turns special values wrong\n");
    ++fails;
  }
  for (int it = 0; it < 100000; ++it) {
    const double d = ldexp((double)(rng() >> 11), -53) * 64.0 - 32.0;  // multiples of 2^-47 in [-32, 32)
    const double k = (double)((long long)(rng() % 64) - 32);
    const unsigned long long a = frac_turns(d), b = frac_turns(d + k);
    const double back = ldexp((double)a, -64);
    const double want = d - std::floor(d);
    if (a != b || std::fabs(back - want) > 1e-15) {
      if (fails++ < 10) printf("frac_turns(%.17g) = %llu\n", d, a);
    }
  }
  printf(fails ? "FAIL %d\n" : "OK\n", fails);
  return fails ? 1 : 0;
}
