/* The float64 log series' quotient s = (m - 1) / (m + 1) as the device forms it
 * (Markstein's method, IBM J. Res. Dev. 34(1), 1990), checked here against the
 * host's correctly rounded division over the reduced range m in
 * [sqrt2 / 2, sqrt2] and its edges, with the initial float reciprocal moved by
 * -K .. K float ulps (the device's approximate reciprocal is within a few).
 * Usage: quotient_check N K [skip_special]; prints "checks differ", exits 1 on
 * any difference. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static uint64_t bits_of(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }
static double from_bits(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }
static float ulps(float f, int k) { uint32_t u; memcpy(&u, &f, 4); u += (uint32_t)k; memcpy(&f, &u, 4); return f; }

static int special = 1;

static double quotient(double a, double d, int k) {
  double y = (double)ulps(1.0f / (float)d, k), e;
  for (int it = 0; it < 3; it++) { /* two Newton steps, then Markstein's reciprocal step */
    e = fma(-d, y, 1.0);
    y = fma(y, e, y);
  }
  if (special && bits_of(d) == 0x3FFFFFFFFFFFFFFFull) y = from_bits(0x3FE0000000000001ull);
  double q = a * y, r;
  for (int it = 0; it < 2; it++) { /* a faithful quotient, then the correctly rounded one */
    r = fma(-d, q, a);
    q = fma(r, y, q);
  }
  return q;
}

static long checks = 0, differ = 0;
static int K = 4;

static void check(double m) {
  const double a = m - 1.0, d = m + 1.0, want = a / d;
  for (int k = -K; k <= K; k++) {
    checks++;
    if (bits_of(quotient(a, d, k)) != bits_of(want) && differ++ < 5)
      printf("m = %a, reciprocal %+d ulps: %a, want %a\n", m, k, quotient(a, d, k), want);
  }
}

int main(int argc, char** argv) {
  const long n = argc > 1 ? atol(argv[1]) : 1000000;
  K = argc > 2 ? atoi(argv[2]) : 4;
  special = !(argc > 3 && atoi(argv[3]));
  const double lo = 0x1.6a09e667f3bcdp-1, hi = 0x1.6a09e667f3bcdp+0;
  uint64_t s = 0x9E3779B97F4A7C15ull;
  for (long i = 0; i < n; i++) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    const double m = from_bits(((s & 1) ? 0x3FF0000000000000ull : 0x3FE0000000000000ull) | (s >> 12));
    if (m >= lo && m <= hi) check(m);
  }
  for (uint64_t j = 0; j < 4096; j++) {
    check(from_bits(0x3FF0000000000000ull + j));
    check(from_bits(0x3FF0000000000000ull - j));
    check(from_bits(bits_of(hi) - j));
    check(from_bits(bits_of(lo) + j));
  }
  check(1.0 - 0x1p-52); /* d = 2 - 2^-52: a significand of all ones */
  check(1.0 - 0x1p-53);
  printf("%ld checks %ld differ\n", checks, differ);
  return differ != 0;
}
