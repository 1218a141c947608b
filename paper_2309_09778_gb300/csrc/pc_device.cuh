// Device-side numerics and shared definitions for the GB300 compressor.
//
// Every floating-point step is an explicit IEEE operation (the library is
// built with --fmad=false; fused multiply-adds appear only where written as
// __fmaf_rn / __fma_rn), so the results are fixed bit for bit by the written
// specification of each step.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pc.h"

namespace pc {

constexpr int kLmax = 24;            // longest Huffman code word
constexpr int kHdr = 256;            // container header bytes
constexpr int kVclamp = 16777215;    // centred predictor inputs clamp to +-(2^24 - 1)
constexpr float kAlpha = 0.0625f;    // leaky ReLU slope 2^-4
constexpr int kMaxH = 64;            // widest hidden layer supported
constexpr int kMaxW = 2048;          // largest weight blob (floats) carried by value
constexpr int kChunkPts = 16384;     // points per pack/decode chunk
constexpr int kBatch = 256;          // SGD minibatch rows

// ---------------------------------------------------------------------------
// Workspace state shared by the kernels of one call.
// ---------------------------------------------------------------------------
struct State {
  // a1: statistics (bit patterns of non-negative magnitudes order like integers)
  unsigned long long amin_bits, amax_bits;
  unsigned int nonfinite, have_normal;
  // a2: constants
  int err;
  int trivial;
  int Kp, Kn, Zq, S;
  float step32, inv32, ebdn32, pad0;
  double stepd, invd, ebdnd;
  double amin, amax;
  // a10-a12: sizes known only on the device
  unsigned int n_used, pad1;
  unsigned long long n_out, total_bits, swords;
  unsigned long long off_cb, off_bb, off_bn, off_ov, off_st, total;
  unsigned long long out_size;
  unsigned int ticket;
  unsigned int pad2[15];
  // a10: first canonical code and first codebook index of every length
  unsigned int cb_first[32], cb_offs[32];
};

// Entries of the FP32 weight blob: W1[h1][k], b1[h1], W2[h2][h1], b2[h2], W3[hl], b3.
__host__ __device__ constexpr int mlp_nweights_c(int k, int h1, int h2) {
  return h1 * k + h1 + (h2 > 0 ? h2 * h1 + h2 : 0) + (h2 > 0 ? h2 : h1) + 1;
}

struct Mlp {
  int k, h1, h2, s_in;
  float w[kMaxW];
};

// ---------------------------------------------------------------------------
// log2 and 2^t, from the mathematics (no vendor math routines).
//
// Single precision uses P. T. P. Tang's table-driven method (ACM TOMS 16(4),
// 1990 for the logarithm; ACM TOMS 15(2), 1989 for the exponential):
//   log2 y = e + LOGR_i + log2(1 + r),  r = fma(m, RCP_i, -1),
//     i = top 7 mantissa bits, c_0 = 1, c_i = 1 + (i + 1/2)/128,
//     RCP_i = float(1/c_i), LOGR_i = float(-log2 RCP_i),
//     log2(1 + r) = r (c1 + r (c2 + r (c3 + r c4))), c_k = (-1)^(k+1)/(k ln 2);
//   2^t = 2^k EXP_j 2^f,  32 k + j = rint(32 t),  2^f = 1 + u + u^2/2 + u^3/6 + u^4/24,
//     u = f ln 2, EXP_j = float(2^(j/32)).
// The tables are generated on the device from the double-precision series
// below (build_tabs) once per call.  Double precision sums the atanh and
// Taylor series directly.
// ---------------------------------------------------------------------------
struct Tabs {
  float rcp[128];
  float logr[128];
  float ex[32];
  float lc[4];
};

__device__ __forceinline__ float pow2_scale_f(int k) { return __uint_as_float((unsigned int)(k + 127) << 23); }

// Exact integer <-> float helpers without conversion instructions: adding
// 1.5 * 2^23 puts rint(u) (round to nearest even, as IEEE addition rounds)
// in the low mantissa bits for |u| < 2^22, and the inverse turns a small
// integer into its float exactly.  Outside that range the conversion
// instructions are used; both give the same values.
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
__device__ __forceinline__ float rint_to_int(float u, int& n) {
  if (fabsf(u) < 4194304.0f) {
    const float t = __fadd_rn(u, kMagic);
    n = __float_as_int(t) - 0x4B400000;
    return __fsub_rn(t, kMagic);
  }
  const float r = rintf(u);
  n = __float2int_rn(r);
  return r;
}
__device__ __forceinline__ float small_int_to_float(int n) {
  if (n > -4194304 && n < 4194304) return __fsub_rn(__int_as_float(n + 0x4B400000), kMagic);
  return __int2float_rn(n);
}

__device__ __forceinline__ float dev_log2f(float y, const Tabs& tb) {
  const unsigned int b = __float_as_uint(y);
  const int e = (int)((b >> 23) & 0xFFu) - 127;
  const int i = (int)((b >> 16) & 0x7Fu);
  const float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
  const float r = __fmaf_rn(m, tb.rcp[i], -1.0f);
  float p = __fmaf_rn(tb.lc[3], r, tb.lc[2]);
  p = __fmaf_rn(p, r, tb.lc[1]);
  p = __fmaf_rn(p, r, tb.lc[0]);
  p = __fmul_rn(p, r);
  const float t = __fadd_rn(tb.logr[i], p);
  return __fadd_rn(__fsub_rn(__int_as_float(e + 0x4B400000), kMagic), t);
}

__device__ __forceinline__ float dev_exp2f(float t, const Tabs& tb) {
  t = fminf(fmaxf(t, -300.0f), 300.0f);
  const float t32 = __fadd_rn(__fmul_rn(t, 32.0f), kMagic);   // |32 t| <= 9600
  const int N = __float_as_int(t32) - 0x4B400000;
  const float nf = __fsub_rn(t32, kMagic);
  const int j = N & 31;
  const int k = (N - j) / 32;
  const float f = __fsub_rn(t, __fmul_rn(nf, 0.03125f));
  const float u = __fmul_rn(f, 0x1.62e430p-1f);
  float p = __fmaf_rn(1.0f / 24.0f, u, 1.0f / 6.0f);
  p = __fmaf_rn(p, u, 0.5f);
  p = __fmaf_rn(p, u, 1.0f);
  p = __fmaf_rn(p, u, 1.0f);
  const float v = __fmul_rn(tb.ex[j], p);
  const int k1 = k / 3;
  const int k2 = (k - k1) / 2;
  const int k3 = k - k1 - k2;
  return __fmul_rn(__fmul_rn(__fmul_rn(v, pow2_scale_f(k1)), pow2_scale_f(k2)), pow2_scale_f(k3));
}

__device__ __forceinline__ double pow2_scale_d(int k) {
  return __longlong_as_double((long long)((unsigned long long)(k + 1023) << 52));
}

// RN(a / d) for the log series' quotient, d = RN(m + 1) in [1.7, 2.42] and
// a = m - 1, by Markstein's method (P. Markstein, IBM J. Res. Dev. 34(1),
// 1990; Cornea, Harrison and Tang, Scientific Computing on Itanium-based
// Systems, 2002), without branches so that the transforms of many points
// overlap on the narrow FP64 pipe:
//  - y: an approximate float reciprocal and two Newton steps, within one ulp
//    of 1/d; one more step on the exact residual 1 - d y gives RN(1/d)
//    (Markstein's reciprocal theorem), except for a significand of all ones,
//    d = 2 - 2^-52 in this range, whose RN(1/d) = 0.5 + 2^-53 is set directly;
//  - q = RN(a y) corrected twice by the exact residual a - d q: the first
//    correction makes q faithful, the second gives RN(a / d) (Markstein's
//    quotient theorem).
__device__ __forceinline__ double div_markstein(double a, double d) {
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__double2float_rn(d)));
  double y = (double)yf;
  double e = __fma_rn(-d, y, 1.0);
  y = __fma_rn(y, e, y);
  e = __fma_rn(-d, y, 1.0);
  y = __fma_rn(y, e, y);
  e = __fma_rn(-d, y, 1.0);
  y = __fma_rn(y, e, y);
  if (__double_as_longlong(d) == 0x3FFFFFFFFFFFFFFFll) y = __longlong_as_double(0x3FE0000000000001ll);
  double q = __dmul_rn(a, y);
  double r = __fma_rn(-d, q, a);
  q = __fma_rn(r, y, q);
  r = __fma_rn(-d, q, a);
  return __fma_rn(r, y, q);
}

// The tests below read the bit pattern (ordered like the value for a
// non-negative double, sign bit set for a negative one) and halve m by its
// exponent (exact): the same results as the floating-point forms, kept off
// the narrow FP64 pipe.
__device__ inline double dev_log2d(double y) {
  const unsigned long long sqrt2_bits = 0x3FF6A09E667F3BCDull;  // 0x1.6a09e667f3bcdp+0
  const double two_over_ln2 = 0x1.71547652b82fep+1;
  int extra = 0;
  if (__double_as_longlong(y) < 0x0010000000000000ll) {  // y < 2^-1022, subnormal: rescale into the normal range
    y = __dmul_rn(y, 0x1p64);
    extra = -64;
  }
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  int e = (int)((b >> 52) & 0x7FFull) - 1023;
  unsigned long long mb = (b & 0xFFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
  if (mb > sqrt2_bits) {  // m > sqrt 2: m / 2
    mb -= 1ull << 52;
    e += 1;
  }
  const double m = __longlong_as_double((long long)mb);
  // 1/(2j+1) for j = 0..10, each rounded once, folded at compile time
  constexpr double inv_odd[11] = {1.0,        1.0 / 3.0,  1.0 / 5.0,  1.0 / 7.0,  1.0 / 9.0, 1.0 / 11.0,
                                  1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0, 1.0 / 21.0};
  double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  double z = __dmul_rn(s, s);
  double p = inv_odd[10];
#pragma unroll
  for (int j = 9; j >= 0; --j) p = __fma_rn(p, z, inv_odd[j]);
  double t = __dmul_rn(__dmul_rn(s, p), two_over_ln2);
  double r = __dadd_rn((double)e, t);
  return extra ? __dadd_rn(r, (double)extra) : r;
}

// dev_log2d for y >= 2^-1022 (or a non-finite y), without branches: the same
// operations and result, with the quotient by div_markstein.
__device__ __forceinline__ double dev_log2d_normal(double y) {
  const unsigned long long sqrt2_bits = 0x3FF6A09E667F3BCDull;  // 0x1.6a09e667f3bcdp+0
  const double two_over_ln2 = 0x1.71547652b82fep+1;
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const bool half = (b & 0xFFFFFFFFFFFFFull) > (sqrt2_bits & 0xFFFFFFFFFFFFFull);  // m > sqrt 2: m / 2
  const int e = (int)((b >> 52) & 0x7FFull) - 1023 + (half ? 1 : 0);
  const double m = __longlong_as_double((long long)((b & 0xFFFFFFFFFFFFFull) | (half ? 0x3FE0000000000000ull
                                                                                        : 0x3FF0000000000000ull)));
  constexpr double inv_odd[11] = {1.0,        1.0 / 3.0,  1.0 / 5.0,  1.0 / 7.0,  1.0 / 9.0, 1.0 / 11.0,
                                  1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0, 1.0 / 21.0};
  const double s = div_markstein(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z = __dmul_rn(s, s);
  double p = inv_odd[10];
#pragma unroll
  for (int j = 9; j >= 0; --j) p = __fma_rn(p, z, inv_odd[j]);
  const double t = __dmul_rn(__dmul_rn(s, p), two_over_ln2);
  return __dadd_rn((double)e, t);
}

__device__ inline double dev_exp2d(double t) {
  const double ln2 = 0x1.62e42fefa39efp-1;
  // 1/i! for i = 0..13: i! is exact in double, so each entry is the division
  // rounded once, folded at compile time (the FP64 pipe is narrow on this part)
  constexpr double inv_fact[14] = {1.0,
                                   1.0,
                                   1.0 / 2.0,
                                   1.0 / 6.0,
                                   1.0 / 24.0,
                                   1.0 / 120.0,
                                   1.0 / 720.0,
                                   1.0 / 5040.0,
                                   1.0 / 40320.0,
                                   1.0 / 362880.0,
                                   1.0 / 3628800.0,
                                   1.0 / 39916800.0,
                                   1.0 / 479001600.0,
                                   1.0 / 6227020800.0};
  if (((unsigned long long)__double_as_longlong(t) & 0x7FFFFFFFFFFFFFFFull) > 0x40A0680000000000ull)  // |t| > 2100
    t = __double_as_longlong(t) < 0 ? -2100.0 : 2100.0;
  double nf = rint(t);
  int k = (int)nf;
  double f = __dsub_rn(t, nf);
  double u = __dmul_rn(f, ln2);
  double p = inv_fact[13];
#pragma unroll
  for (int i = 12; i >= 0; --i) p = __fma_rn(p, u, inv_fact[i]);
  int k1 = k / 3;
  int k2 = (k - k1) / 2;
  int k3 = k - k1 - k2;
  return __dmul_rn(__dmul_rn(__dmul_rn(p, pow2_scale_d(k1)), pow2_scale_d(k2)), pow2_scale_d(k3));
}

// Table generation: entry i is computed by thread i of the calling block.
__device__ inline void build_tabs_entry(Tabs* tb, int i) {
  if (i < 128) {
    const double c = i == 0 ? 1.0 : 1.0 + ((double)i + 0.5) / 128.0;
    const float r = __double2float_rn(__ddiv_rn(1.0, c));
    tb->rcp[i] = r;
    tb->logr[i] = __double2float_rn(-dev_log2d((double)r));
  }
  if (i < 32) tb->ex[i] = __double2float_rn(dev_exp2d((double)i / 32.0));
  if (i < 4) {
    const double ln2 = 0x1.62e42fefa39efp-1;
    const double v = i == 0 ? __ddiv_rn(1.0, ln2)
                            : (i == 1 ? __ddiv_rn(-1.0, 2.0 * ln2)
                                      : (i == 2 ? __ddiv_rn(1.0, 3.0 * ln2) : __ddiv_rn(-1.0, 4.0 * ln2)));
    tb->lc[i] = __double2float_rn(v);
  }
}

// ---------------------------------------------------------------------------
// Transform (Eq. 6, 7, 12) and its inverse.  Code classes: q <= Zq is zero,
// Zq < q <= S positive, q > S negative.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int code_class(int q, const State& c) { return q <= c.Zq ? 0 : (q <= c.S ? 1 : 2); }

template <typename T> struct Num;

template <> struct Num<float> {
  static __device__ __forceinline__ float recon(int q, const State& c, const Tabs& tb) {
    const int cl = code_class(q, c);
    if (cl == 0) return 0.0f;
    const int n = q - (cl == 1 ? c.Kp : c.Kn);
    const float a = dev_exp2f(__fmul_rn(small_int_to_float(n), c.step32), tb);
    return cl == 1 ? a : -a;
  }
  // code of x and whether it reproduces x within the bound
  static __device__ __forceinline__ int transform(float x, const State& c, const Tabs& tb, bool& ok) {
    const unsigned int b = __float_as_uint(x);
    const float a = fabsf(x);
    if (b == 0u) { ok = true; return c.Zq; }
    if (a < 0x1p-126f) { ok = false; return c.Zq; }
    const float l = dev_log2f(a, tb);
    int n;
    const float nf = rint_to_int(__fmul_rn(l, c.inv32), n);
    const bool pos = x > 0.0f;
    const int q = n + (pos ? c.Kp : c.Kn);
    if (code_class(q, c) != (pos ? 1 : 2)) { ok = false; return q; }
    const float r = dev_exp2f(__fmul_rn(nf, c.step32), tb);
    const float err = fabsf(__fsub_rn(r, a));
    ok = err <= __fmul_rd(c.ebdn32, a);  // exact: a <= RD(p) iff a <= p for a float a
    return q;
  }
};

template <> struct Num<double> {
  static __device__ __forceinline__ double recon(int q, const State& c, const Tabs&) {
    int cl = code_class(q, c);
    if (cl == 0) return 0.0;
    int n = q - (cl == 1 ? c.Kp : c.Kn);
    double a = dev_exp2d(__dmul_rn((double)n, c.stepd));
    return cl == 1 ? a : -a;
  }
  // Without branches: every case computes the whole chain (on a stand-in
  // for zero and subnormal magnitudes) and selects its result.
  static __device__ __forceinline__ int transform(double x, const State& c, const Tabs&, bool& ok) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long ab = b & 0x7FFFFFFFFFFFFFFFull;
    const bool zero = b == 0ull;                          // +0.0 only
    const bool small = ab < 0x0010000000000000ull;        // |x| < 2^-1022 (and -0.0)
    const double a = __longlong_as_double((long long)(small ? 0x3FF0000000000000ull : ab));
    const double l = dev_log2d_normal(a);
    const double nf = rint(__dmul_rn(l, c.invd));
    const int n = (int)nf;
    const bool pos = x > 0.0;
    const int q = n + (pos ? c.Kp : c.Kn);
    const bool cls = code_class(q, c) == (pos ? 1 : 2);
    const double r = dev_exp2d(__dmul_rn((double)n, c.stepd));
    const double err = fabs(__dsub_rn(r, a));
    const bool in_bound = err <= __dmul_rd(c.ebdnd, a);
    ok = zero || (!small && cls && in_bound);
    return small ? c.Zq : q;
  }
};

// ---------------------------------------------------------------------------
// Stencils.  S7: the 3-D Lorenzo set; S13: every (dz,dy,dx) in {-1,0,1}^3 that
// precedes (0,0,0) in raster order.  Lorenzo weights are the SZ formula's signs
// (+1 for an odd number of non-zero offsets, -1 for an even number).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int s7_dz(int i) { return (i == 0 || i == 3 || i == 4 || i == 6) ? -1 : 0; }
__host__ __device__ constexpr int s7_dy(int i) { return (i == 1 || i == 3 || i == 5 || i == 6) ? -1 : 0; }
__host__ __device__ constexpr int s7_dx(int i) { return (i == 2 || i == 4 || i == 5 || i == 6) ? -1 : 0; }
__host__ __device__ constexpr int s13_dz(int i) { return i < 9 ? -1 : 0; }
__host__ __device__ constexpr int s13_dy(int i) { return i < 9 ? (i / 3) - 1 : (i < 12 ? -1 : 0); }
__host__ __device__ constexpr int s13_dx(int i) { return i < 9 ? (i % 3) - 1 : (i < 12 ? (i - 9) - 1 : -1); }
__host__ __device__ constexpr int st_dz(int k, int i) { return k == 7 ? s7_dz(i) : s13_dz(i); }
__host__ __device__ constexpr int st_dy(int k, int i) { return k == 7 ? s7_dy(i) : s13_dy(i); }
__host__ __device__ constexpr int st_dx(int k, int i) { return k == 7 ? s7_dx(i) : s13_dx(i); }
__host__ __device__ constexpr int lz_w(int k, int i) {
  return (st_dz(k, i) > 0 || st_dy(k, i) > 0 || st_dx(k, i) > 0)
             ? 0
             : ((((st_dz(k, i) != 0) + (st_dy(k, i) != 0) + (st_dx(k, i) != 0)) & 1) ? 1 : -1);
}

__device__ __forceinline__ int clampv(long long v) {
  return (int)(v > kVclamp ? kVclamp : (v < -kVclamp ? -kVclamp : v));
}
// the same clamp for a difference of two codes, both within +-2^30
__device__ __forceinline__ int clampd(int q, int da) { return min(max(q - da, -kVclamp), kVclamp); }

__device__ __forceinline__ int bitlen_u(unsigned int a) { return 32 - __clz(a); }

// Perceptron forward (Section IV.B) in FP32 with the stated operation order:
// u_i = v_i 2^-s; each unit starts at its bias and accumulates fma(w, u_i, acc)
// over inputs in order; leaky ReLU on hidden units; linear output scaled by 2^s.
template <int K, int H1, int H2>
__device__ __forceinline__ float mlp_fwd(const Mlp& m, const int* v, float sig, float unsig) {
  float u[K];
#pragma unroll
  for (int i = 0; i < K; ++i) u[i] = __fmul_rn(__int2float_rn(v[i]), sig);
  float a1[H1];
#pragma unroll
  for (int j = 0; j < H1; ++j) {
    float acc = m.w[H1 * K + j];
#pragma unroll
    for (int i = 0; i < K; ++i) acc = __fmaf_rn(m.w[j * K + i], u[i], acc);
    a1[j] = acc >= 0.0f ? acc : __fmul_rn(acc, kAlpha);
  }
  constexpr int P2 = H1 * K + H1;
  if constexpr (H2 > 0) {
    float a2[H2];
#pragma unroll
    for (int j = 0; j < H2; ++j) {
      float acc = m.w[P2 + H2 * H1 + j];
#pragma unroll
      for (int i = 0; i < H1; ++i) acc = __fmaf_rn(m.w[P2 + j * H1 + i], a1[i], acc);
      a2[j] = acc >= 0.0f ? acc : __fmul_rn(acc, kAlpha);
    }
    constexpr int P3 = P2 + H2 * H1 + H2;
    float o = m.w[P3 + H2];
#pragma unroll
    for (int j = 0; j < H2; ++j) o = __fmaf_rn(m.w[P3 + j], a2[j], o);
    return __fmul_rn(o, unsig);
  } else {
    float o = m.w[P2 + H1];
#pragma unroll
    for (int j = 0; j < H1; ++j) o = __fmaf_rn(m.w[P2 + j], a1[j], o);
    return __fmul_rn(o, unsig);
  }
}

// Two points at once through the same perceptron, on the packed two-lane
// fp32 operations (__ffma2_rn, __fmul2_rn): each lane performs the correctly
// rounded IEEE operation of the scalar form, so both results equal
// mlp_fwd's bit for bit while the instruction count nearly halves.  The
// leaky ReLU is max(v, alpha v), the same value as the scalar select for
// every v (alpha > 0; a zero keeps its sign).
__device__ __forceinline__ float2 f2_leaky(float2 v) {
  const float2 m = __fmul2_rn(v, make_float2(kAlpha, kAlpha));
  return make_float2(fmaxf(v.x, m.x), fmaxf(v.y, m.y));
}

template <int K, int H1, int H2, typename WF>
__device__ __forceinline__ void mlp_fwd2_core(WF W, const int* va, const int* vb, float sig, float unsig, float& pa,
                                              float& pb) {
  float2 u[K];
#pragma unroll
  for (int i = 0; i < K; ++i)
    u[i] = make_float2(__fmul_rn(__int2float_rn(va[i]), sig), __fmul_rn(__int2float_rn(vb[i]), sig));
  float2 a1[H1];
#pragma unroll
  for (int j = 0; j < H1; ++j) {
    float2 acc = W(H1 * K + j);
#pragma unroll
    for (int i = 0; i < K; ++i) acc = __ffma2_rn(W(j * K + i), u[i], acc);
    a1[j] = f2_leaky(acc);
  }
  constexpr int P2 = H1 * K + H1;
  float2 o;
  if constexpr (H2 > 0) {
    float2 a2[H2];
#pragma unroll
    for (int j = 0; j < H2; ++j) {
      float2 acc = W(P2 + H2 * H1 + j);
#pragma unroll
      for (int i = 0; i < H1; ++i) acc = __ffma2_rn(W(P2 + j * H1 + i), a1[i], acc);
      a2[j] = f2_leaky(acc);
    }
    constexpr int P3 = P2 + H2 * H1 + H2;
    o = W(P3 + H2);
#pragma unroll
    for (int j = 0; j < H2; ++j) o = __ffma2_rn(W(P3 + j), a2[j], o);
  } else {
    o = W(P2 + H1);
#pragma unroll
    for (int j = 0; j < H1; ++j) o = __ffma2_rn(W(P2 + j), a1[j], o);
  }
  o = __fmul2_rn(o, make_float2(unsig, unsig));
  pa = o.x;
  pb = o.y;
}

// Weights from the kernel parameters (constant bank).
template <int K, int H1, int H2>
__device__ __forceinline__ void mlp_fwd2(const Mlp& m, const int* va, const int* vb, float sig, float unsig, float& pa,
                                         float& pb) {
  mlp_fwd2_core<K, H1, H2>([&](int idx) { return make_float2(m.w[idx], m.w[idx]); }, va, vb, sig, unsig, pa, pb);
}

// Runtime-shaped forward for widths without a compiled instance.
__device__ __forceinline__ float mlp_fwd_rt(const Mlp& m, const int* v, float sig, float unsig) {
  const int K = m.k, H1 = m.h1, H2 = m.h2;
  float u[13];
  for (int i = 0; i < K; ++i) u[i] = __fmul_rn(__int2float_rn(v[i]), sig);
  float a1[kMaxH], a2[kMaxH];
  for (int j = 0; j < H1; ++j) {
    float acc = m.w[H1 * K + j];
    for (int i = 0; i < K; ++i) acc = __fmaf_rn(m.w[j * K + i], u[i], acc);
    a1[j] = acc >= 0.0f ? acc : __fmul_rn(acc, kAlpha);
  }
  int p = H1 * K + H1;
  const float* hl = a1;
  int nl = H1;
  if (H2 > 0) {
    for (int j = 0; j < H2; ++j) {
      float acc = m.w[p + H2 * H1 + j];
      for (int i = 0; i < H1; ++i) acc = __fmaf_rn(m.w[p + j * H1 + i], a1[i], acc);
      a2[j] = acc >= 0.0f ? acc : __fmul_rn(acc, kAlpha);
    }
    p += H2 * H1 + H2;
    hl = a2;
    nl = H2;
  }
  float o = m.w[p + nl];
  for (int j = 0; j < nl; ++j) o = __fmaf_rn(m.w[p + j], hl[j], o);
  return __fmul_rn(o, unsig);
}

__device__ __forceinline__ int round_pred(float p) {
  if (p != p) return 0;
  p = fminf(fmaxf(p, -1073741824.0f), 1073741824.0f);
  return __float2int_rn(p);
}

}  // namespace pc
