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
};

struct Mlp {
  int k, h1, h2, s_in;
  float w[kMaxW];
};

// ---------------------------------------------------------------------------
// log2 and 2^t.  Series from the mathematics: ln y = 2 atanh((y-1)/(y+1)) with
// atanh s = s + s^3/3 + s^5/5 + ...; 2^f = exp(f ln 2) by its Taylor series.
// Both run Horner's rule with fused multiply-adds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dev_log2f(float y) {
  const float sqrt2 = 0x1.6a09e6p+0f;   // sqrt(2) rounded to float
  const float two_over_ln2 = 0x1.715476p+1f;
  unsigned int b = __float_as_uint(y);
  int e = (int)((b >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
  if (m > sqrt2) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  float z = __fmul_rn(s, s);
  float p = 1.0f / 9.0f;
  p = __fmaf_rn(p, z, 1.0f / 7.0f);
  p = __fmaf_rn(p, z, 1.0f / 5.0f);
  p = __fmaf_rn(p, z, 1.0f / 3.0f);
  p = __fmaf_rn(p, z, 1.0f);
  float t = __fmul_rn(__fmul_rn(s, p), two_over_ln2);
  return __fadd_rn(__int2float_rn(e), t);
}

__device__ __forceinline__ float pow2_scale_f(int k) { return __uint_as_float((unsigned int)(k + 127) << 23); }

__device__ __forceinline__ float dev_exp2f(float t) {
  const float ln2 = 0x1.62e430p-1f;
  t = fminf(fmaxf(t, -300.0f), 300.0f);
  float nf = rintf(t);
  int k = __float2int_rn(nf);
  float f = __fsub_rn(t, nf);
  float u = __fmul_rn(f, ln2);
  float p = 1.0f / 5040.0f;
  p = __fmaf_rn(p, u, 1.0f / 720.0f);
  p = __fmaf_rn(p, u, 1.0f / 120.0f);
  p = __fmaf_rn(p, u, 1.0f / 24.0f);
  p = __fmaf_rn(p, u, 1.0f / 6.0f);
  p = __fmaf_rn(p, u, 0.5f);
  p = __fmaf_rn(p, u, 1.0f);
  p = __fmaf_rn(p, u, 1.0f);
  int k1 = k / 3;
  int k2 = (k - k1) / 2;
  int k3 = k - k1 - k2;
  return __fmul_rn(__fmul_rn(__fmul_rn(p, pow2_scale_f(k1)), pow2_scale_f(k2)), pow2_scale_f(k3));
}

__device__ __forceinline__ double pow2_scale_d(int k) {
  return __longlong_as_double((long long)((unsigned long long)(k + 1023) << 52));
}

__device__ inline double dev_log2d(double y) {
  const double sqrt2 = 0x1.6a09e667f3bcdp+0;
  const double two_over_ln2 = 0x1.71547652b82fep+1;
  int extra = 0;
  if (y < 0x1p-1022) {  // subnormal: rescale into the normal range
    y = __dmul_rn(y, 0x1p64);
    extra = -64;
  }
  unsigned long long b = (unsigned long long)__double_as_longlong(y);
  int e = (int)((b >> 52) & 0x7FFull) - 1023;
  double m = __longlong_as_double((long long)((b & 0xFFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
  if (m > sqrt2) {
    m = __dmul_rn(m, 0.5);
    e += 1;
  }
  double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  double z = __dmul_rn(s, s);
  double p = 1.0 / 21.0;
#pragma unroll
  for (int j = 9; j >= 0; --j) p = __fma_rn(p, z, 1.0 / (double)(2 * j + 1));
  double t = __dmul_rn(__dmul_rn(s, p), two_over_ln2);
  double r = __dadd_rn((double)e, t);
  return extra ? __dadd_rn(r, (double)extra) : r;
}

__device__ inline double dev_exp2d(double t) {
  const double ln2 = 0x1.62e42fefa39efp-1;
  // 1/i! for i = 0..13, each the division 1/i! with i! exact in double
  t = fmin(fmax(t, -2100.0), 2100.0);
  double nf = rint(t);
  int k = (int)nf;
  double f = __dsub_rn(t, nf);
  double u = __dmul_rn(f, ln2);
  double fact = 6227020800.0;  // 13!
  double p = __ddiv_rn(1.0, fact);
#pragma unroll
  for (int i = 12; i >= 0; --i) {
    fact = fact / (double)(i + 1);  // exact: i! is an integer below 2^53
    p = __fma_rn(p, u, __ddiv_rn(1.0, fact));
  }
  int k1 = k / 3;
  int k2 = (k - k1) / 2;
  int k3 = k - k1 - k2;
  return __dmul_rn(__dmul_rn(__dmul_rn(p, pow2_scale_d(k1)), pow2_scale_d(k2)), pow2_scale_d(k3));
}

// ---------------------------------------------------------------------------
// Transform (Eq. 6, 7, 12) and its inverse.  Code classes: q <= Zq is zero,
// Zq < q <= S positive, q > S negative.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int code_class(int q, const State& c) { return q <= c.Zq ? 0 : (q <= c.S ? 1 : 2); }

template <typename T> struct Num;

template <> struct Num<float> {
  static __device__ __forceinline__ float recon(int q, const State& c) {
    int cl = code_class(q, c);
    if (cl == 0) return 0.0f;
    int n = q - (cl == 1 ? c.Kp : c.Kn);
    float a = dev_exp2f(__fmul_rn(__int2float_rn(n), c.step32));
    return cl == 1 ? a : -a;
  }
  // code of x and whether it reproduces x within the bound
  static __device__ __forceinline__ int transform(float x, const State& c, bool& ok) {
    unsigned int b = __float_as_uint(x);
    float a = fabsf(x);
    if (b == 0u) { ok = true; return c.Zq; }
    if (a < 0x1p-126f) { ok = false; return c.Zq; }
    float l = dev_log2f(a);
    float nf = rintf(__fmul_rn(l, c.inv32));
    int n = __float2int_rn(nf);
    bool pos = x > 0.0f;
    int q = n + (pos ? c.Kp : c.Kn);
    if (code_class(q, c) != (pos ? 1 : 2)) { ok = false; return q; }
    float r = dev_exp2f(__fmul_rn(__int2float_rn(n), c.step32));
    float err = fabsf(__fsub_rn(r, a));
    ok = err <= __fmul_rd(c.ebdn32, a);  // exact: a <= RD(p) iff a <= p for a float a
    return q;
  }
  static __device__ __forceinline__ bool is_normal_mag(float a) { return a >= 0x1p-126f; }
};

template <> struct Num<double> {
  static __device__ __forceinline__ double recon(int q, const State& c) {
    int cl = code_class(q, c);
    if (cl == 0) return 0.0;
    int n = q - (cl == 1 ? c.Kp : c.Kn);
    double a = dev_exp2d(__dmul_rn((double)n, c.stepd));
    return cl == 1 ? a : -a;
  }
  static __device__ __forceinline__ int transform(double x, const State& c, bool& ok) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    double a = fabs(x);
    if (b == 0ull) { ok = true; return c.Zq; }
    if (a < 0x1p-1022) { ok = false; return c.Zq; }
    double l = dev_log2d(a);
    double nf = rint(__dmul_rn(l, c.invd));
    int n = (int)nf;
    bool pos = x > 0.0;
    int q = n + (pos ? c.Kp : c.Kn);
    if (code_class(q, c) != (pos ? 1 : 2)) { ok = false; return q; }
    double r = dev_exp2d(__dmul_rn((double)n, c.stepd));
    double err = fabs(__dsub_rn(r, a));
    ok = err <= __dmul_rd(c.ebdnd, a);
    return q;
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
