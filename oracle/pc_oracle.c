/*
 * CPU oracle for the perceptron-predicted, pointwise-relative-error-bounded
 * compressor of arXiv 2309.09778.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * The functions follow the paper's steps in its order:
 *   Section III   relative -> absolute (log) map with sign factors, Eq. 6-12
 *   Section IV.A  Lorenzo prediction surface (the SZ prediction formula)
 *   Section IV.B  three-layer perceptron with leaky ReLU, Lorenzo-aligned init
 *   Section IV.C  sampled training, 8:2 split, L2 term, several (lr, lambda)
 *   Section IV.D  data selection from (pre-quantized) true values; balance points
 *   Section V     Algorithm 1 (compression) and the decompression procedure
 * Where the paper is silent the stated readings are marked "Reading:".
 *
 * Parity status: every function is pinned by the tests against closed forms,
 * brute force or library routines, except the paper-level compression-ratio
 * claim (Section VI), which needs the SEG-Y data and SZ2.1: parity unpinned.
 */
#include "pc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Our own log2 / exp2.  From the mathematics, not from any vendor library.  */
/*                                                                           */
/* Single precision follows the table-driven method of P. T. P. Tang        */
/* ("Table-driven implementation of the logarithm function in IEEE           */
/* floating-point arithmetic", ACM TOMS 16(4), 1990; "... exponential        */
/* function ...", ACM TOMS 15(2), 1989):                                     */
/*   log2 y = e + log2 m, m in [1,2) split as m = c_i (1 + r): i = top 7     */
/*   mantissa bits, c_0 = 1, c_i = 1 + (i + 1/2)/128, RCP_i = (float)(1/c_i) */
/*   (double division, then rounding), r = fma(m, RCP_i, -1), and             */
/*   log2 m = LOGR_i + log2(1 + r) with LOGR_i = (float)(-log2 RCP_i) from     */
/*   our double log2; log2(1 + r) = r (c1 + r (c2 + r (c3 + r c4))),         */
/*   c_k = (-1)^(k+1) / (k ln 2) rounded to float.                           */
/*   2^t = 2^k 2^(j/32) 2^f with 32k + j = rint(32 t), |f| <= 1/64;           */
/*   2^f = 1 + u + u^2/2 + u^3/6 + u^4/24, u = f ln 2; EXP_j = (float)2^(j/32)*/
/*   from our double exp2.                                                   */
/* Double precision sums the atanh and Taylor series directly.              */
/* ------------------------------------------------------------------------- */

static const double O_SQRT2_D = 0x1.6a09e667f3bcdp+0;
static const double O_2LN2_D = 0x1.71547652b82fep+1;
static const double O_LN2_D = 0x1.62e42fefa39efp-1;

static float f_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_of_f(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }
static double d_from_bits(uint64_t b) { double f; memcpy(&f, &b, 8); return f; }
static uint64_t bits_of_d(double f) { uint64_t b; memcpy(&b, &f, 8); return b; }

double orc_L64(double y);
double orc_E64(double t);

static float o_rcp[128], o_logr[128], o_exp[32];
static float o_lc[4];
static int o_tab_ready = 0;

static void o_tables(void) {
  if (o_tab_ready) return;
  for (int i = 0; i < 128; i++) {
    double c = i == 0 ? 1.0 : 1.0 + ((double)i + 0.5) / 128.0;
    o_rcp[i] = (float)(1.0 / c);
    o_logr[i] = (float)(-orc_L64((double)o_rcp[i]));
  }
  for (int j = 0; j < 32; j++) o_exp[j] = (float)orc_E64((double)j / 32.0);
  double ln2 = O_LN2_D;
  o_lc[0] = (float)(1.0 / ln2);
  o_lc[1] = (float)(-1.0 / (2.0 * ln2));
  o_lc[2] = (float)(1.0 / (3.0 * ln2));
  o_lc[3] = (float)(-1.0 / (4.0 * ln2));
  o_tab_ready = 1;
}

/* log2 of a positive normal float. */
float orc_L32(float y) {
  o_tables();
  uint32_t b = bits_of_f(y);
  int e = (int)((b >> 23) & 0xFFu) - 127;
  int i = (int)((b >> 16) & 0x7Fu);
  float m = f_from_bits((b & 0x7FFFFFu) | 0x3F800000u); /* [1, 2) */
  float r = fmaf(m, o_rcp[i], -1.0f);
  float p = fmaf(o_lc[3], r, o_lc[2]);
  p = fmaf(p, r, o_lc[1]);
  p = fmaf(p, r, o_lc[0]);
  p = p * r;
  float t = o_logr[i] + p;
  return (float)e + t;
}

/* 2^t for finite t (clamped to [-300, 300]). */
float orc_E32(float t) {
  o_tables();
  if (t > 300.0f) t = 300.0f;
  if (t < -300.0f) t = -300.0f;
  float nf = rintf(t * 32.0f);
  int N = (int)nf;
  int j = N & 31;
  int k = (N - j) / 32;
  float f = t - nf * 0.03125f;
  float u = f * 0x1.62e430p-1f;
  float p = fmaf(1.0f / 24.0f, u, 1.0f / 6.0f);
  p = fmaf(p, u, 0.5f);
  p = fmaf(p, u, 1.0f);
  p = fmaf(p, u, 1.0f);
  float v = o_exp[j] * p;
  int k1 = k / 3;
  int k2 = (k - k1) / 2;
  int k3 = k - k1 - k2;
  float s1 = f_from_bits((uint32_t)(k1 + 127) << 23);
  float s2 = f_from_bits((uint32_t)(k2 + 127) << 23);
  float s3 = f_from_bits((uint32_t)(k3 + 127) << 23);
  return ((v * s1) * s2) * s3;
}

/* log2 of a positive double (subnormals are rescaled first): atanh series. */
double orc_L64(double y) {
  if (y < 0x1p-1022) return orc_L64(y * 0x1p64) - 64.0;
  uint64_t b = bits_of_d(y);
  int e = (int)((b >> 52) & 0x7FFu) - 1023;
  double m = d_from_bits((b & 0xFFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
  if (m > O_SQRT2_D) { m = m * 0.5; e = e + 1; }
  double s = (m - 1.0) / (m + 1.0);
  double z = s * s;
  double p = 1.0 / 21.0;
  for (int j = 9; j >= 0; j--) p = fma(p, z, 1.0 / (double)(2 * j + 1));
  double t = s * p;
  t = t * O_2LN2_D;
  return (double)e + t;
}

/* 2^t for finite t (clamped to [-2100, 2100]). */
double orc_E64(double t) {
  if (t > 2100.0) t = 2100.0;
  if (t < -2100.0) t = -2100.0;
  double nf = rint(t);
  int k = (int)nf;
  double f = t - nf;
  double u = f * O_LN2_D;
  /* coefficients 1/i! for i = 13 .. 0 */
  double fact[14];
  fact[0] = 1.0;
  for (int i = 1; i < 14; i++) fact[i] = fact[i - 1] * (double)i;
  double p = 1.0 / fact[13];
  for (int i = 12; i >= 0; i--) p = fma(p, u, 1.0 / fact[i]);
  int k1 = k / 3;
  int k2 = (k - k1) / 2;
  int k3 = k - k1 - k2;
  double s1 = d_from_bits((uint64_t)(k1 + 1023) << 52);
  double s2 = d_from_bits((uint64_t)(k2 + 1023) << 52);
  double s3 = d_from_bits((uint64_t)(k3 + 1023) << 52);
  return ((p * s1) * s2) * s3;
}

/* ------------------------------------------------------------------------- */
/* Counter-based hash (SplitMix64 finaliser, Steele, Lea & Flood, OOPSLA     */
/* 2014) and CRC-32 (IEEE 802.3 polynomial, reflected, bitwise).             */
/* ------------------------------------------------------------------------- */
uint64_t orc_mix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint32_t orc_crc32(const uint8_t* p, size_t n) {
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; i++) {
    c ^= p[i];
    for (int k = 0; k < 8; k++) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
  }
  return c ^ 0xFFFFFFFFu;
}

/* ------------------------------------------------------------------------- */
/* Step a1: global statistics (Algorithm 1 input "max/min of the dataset").  */
/* abs_min is the non-zero minimum absolute value (Section III.B).           */
/* Reading: subnormal magnitudes are left out of abs_min (they become        */
/* balance points); NaN/Inf are rejected.                                    */
/* ------------------------------------------------------------------------- */
int orc_stats(const void* x, uint64_t n, int dtype, double* amin, double* amax, int* trivial) {
  double mn = INFINITY, mx = 0.0;
  int have = 0;
  for (uint64_t i = 0; i < n; i++) {
    double a;
    if (dtype == ORC_F32) {
      float v = ((const float*)x)[i];
      if (!isfinite(v)) return ORC_ERR_NONFINITE;
      a = fabs((double)v);
      if (a >= 0x1p-126) { have = 1; if (a < mn) mn = a; }
    } else if (dtype == ORC_F64) {
      double v = ((const double*)x)[i];
      if (!isfinite(v)) return ORC_ERR_NONFINITE;
      a = fabs(v);
      if (a >= 0x1p-1022) { have = 1; if (a < mn) mn = a; }
    } else {
      return ORC_ERR_DTYPE;
    }
    if (a > mx) mx = a;
  }
  if (!have) { mn = 1.0; mx = 1.0; }
  *amin = mn;
  *amax = mx;
  *trivial = !have;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Step a2: constants.                                                        */
/*   b_a = log2(1 + eb)                                   (Eq. 8, Alg. 1)    */
/*   factor_pos = abs_min                                  (Eq. 9)            */
/*   log2 factor_neg = log2(abs_max + e0) + log2 factor_pos                   */
/*                     + 2 log2(1 + eb) - log2(abs_min - e0)  (Eq. 10/11)     */
/*   zero image f(e0 * factor_pos)                         (Eq. 12)           */
/*   sign boundary f((abs_max + e0) factor_pos) + g(eb)    (Section III.B)    */
/* Reading: e0 is the smallest positive representable value of the dtype.    */
/* Reading: the log of a product is taken as the sum of logs, and each        */
/* factor's log is rounded to a whole number K of quantization steps 2 b_a.  */
/* By Eq. 5 this is the same as using the constant 2^(K 2 b_a) as the factor. */
/* In code units (one unit = 2 b_a): positive image q = n + Kp, negative      */
/* image q = n + Kn, zero image Zq, with n = rint(log2|x| / (2 b_a)).         */
/* ------------------------------------------------------------------------- */
int orc_make_consts(int dtype, double amin, double amax, int trivial, double eb, orc_consts* c) {
  if (!(eb > 0.0 && eb < 1.0)) return ORC_ERR_ARG;
  if (dtype != ORC_F32 && dtype != ORC_F64) return ORC_ERR_DTYPE;
  memset(c, 0, sizeof(*c));
  c->dtype = dtype;
  c->eb = eb;
  c->abs_min = amin;
  c->abs_max = amax;
  c->trivial = trivial;
  double e0 = dtype == ORC_F32 ? 0x1p-149 : 0x1p-1074;
  double le0 = dtype == ORC_F32 ? -149.0 : -1074.0;  /* log2 e0, exact */
  double ba = orc_L64(1.0 + eb);
  double step = ba + ba;
  c->step64 = step;
  double kp = rint(orc_L64(amin) / step);
  double lfn = ((orc_L64(amax + e0) + orc_L64(amin)) + step) - orc_L64(amin - e0);
  double kn = rint(lfn / step);
  double zq = rint(le0 / step) + kp;
  double s = rint(orc_L64(amax + e0) / step) + kp;
  double span = (dtype == ORC_F32 ? 151.0 : 1076.0) / step + 2.0;
  double lim = 1073741824.0; /* 2^30 */
  if (fabs(kp) + span > lim || fabs(kn) + span > lim || fabs(zq) > lim || fabs(s) > lim)
    return ORC_ERR_EB_RANGE;
  c->Kp = (int32_t)kp;
  c->Kn = (int32_t)kn;
  c->Zq = (int32_t)zq;
  c->S = (int32_t)s;
  c->step32 = (float)step;
  c->inv32 = 1.0f / c->step32;
  float ef = (float)eb;
  if ((double)ef > eb) ef = nextafterf(ef, 0.0f);
  c->ebdn32 = ef;
  c->stepd = step;
  c->invd = 1.0 / step;
  c->ebdnd = eb;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Step a4 and its inverse (Eq. 6, 7, 12 and the inverse map, Section III.B).*/
/* Class of a code: q <= Zq zero, Zq < q <= S positive, q > S negative.       */
/* Reading: Alg. 1 multiplies a negative value by factor_neg; with Eq. 7 this */
/* is |x| * factor_neg.  Reading: only +0.0 maps to the zero image; -0.0,     */
/* subnormals and any point whose code does not reproduce it within the bound */
/* are forced balance points (stored verbatim).                              */
/* ------------------------------------------------------------------------- */
static int o_class(int32_t q, const orc_consts* c) { return q <= c->Zq ? 0 : (q <= c->S ? 1 : 2); }

float orc_recon32(int32_t q, const orc_consts* c) {
  int cl = o_class(q, c);
  if (cl == 0) return 0.0f;
  int32_t n = q - (cl == 1 ? c->Kp : c->Kn);
  float t = (float)n * c->step32;
  float a = orc_E32(t);
  return cl == 1 ? a : -a;
}

double orc_recon64(int32_t q, const orc_consts* c) {
  int cl = o_class(q, c);
  if (cl == 0) return 0.0;
  int32_t n = q - (cl == 1 ? c->Kp : c->Kn);
  double t = (double)n * c->stepd;
  double a = orc_E64(t);
  return cl == 1 ? a : -a;
}

void orc_transform32(float x, const orc_consts* c, int32_t* dq, int* ok) {
  uint32_t b = bits_of_f(x);
  float a = fabsf(x);
  if (b == 0u) { *dq = c->Zq; *ok = 1; return; }
  if (a < 0x1p-126f) { *dq = c->Zq; *ok = 0; return; }
  float l = orc_L32(a);
  float nf = rintf(l * c->inv32);
  int32_t n = (int32_t)nf;
  int32_t q = n + (x > 0.0f ? c->Kp : c->Kn);
  *dq = q;
  if (o_class(q, c) != (x > 0.0f ? 1 : 2)) { *ok = 0; return; }
  float r = orc_E32((float)n * c->step32);
  float err = fabsf(r - a);
  /* err <= eb * |x| decided exactly: the product of two floats is exact in double. */
  *ok = (double)err <= (double)c->ebdn32 * (double)a;
}

void orc_transform64(double x, const orc_consts* c, int32_t* dq, int* ok) {
  uint64_t b = bits_of_d(x);
  double a = fabs(x);
  if (b == 0u) { *dq = c->Zq; *ok = 1; return; }
  if (a < 0x1p-1022) { *dq = c->Zq; *ok = 0; return; }
  double l = orc_L64(a);
  double nf = rint(l * c->invd);
  int32_t n = (int32_t)nf;
  int32_t q = n + (x > 0.0 ? c->Kp : c->Kn);
  *dq = q;
  if (o_class(q, c) != (x > 0.0 ? 1 : 2)) { *ok = 0; return; }
  double r = orc_E64((double)n * c->stepd);
  double err = fabs(r - a);
  /* exact product in binary128 (113-bit significand holds 53 x 53 bits) */
  _Float128 prod = (_Float128)c->ebdnd * (_Float128)a;
  *ok = (_Float128)err <= prod;
}

/* ------------------------------------------------------------------------- */
/* Blocks, stencils and predictors (Section IV.A, IV.B, IV.D).               */
/* Blocks tile the field from the origin; edge blocks are truncated.  The    */
/* block anchor (local origin) is a balance point (Section IV.D.2).  The     */
/* predictor reads the exact pre-quantized codes of causal in-block          */
/* neighbours, centred on the anchor; a neighbour outside the block reads 0. */
/* Reading: the "true values" of the modified selection rule are the          */
/* pre-quantized codes, which the decoder reproduces exactly, so there is no  */
/* drift and compression is fully parallel.                                  */
/* ------------------------------------------------------------------------- */
#define O_VCLAMP 16777215  /* 2^24 - 1 */
static const int O_S7[7][3] = {{-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {-1, -1, 0},
                               {-1, 0, -1}, {0, -1, -1}, {-1, -1, -1}};
static const int O_LZ7[7] = {1, 1, 1, -1, -1, -1, 1};

static void o_stencil(int k, int i, int* dz, int* dy, int* dx) {
  if (k == 7) { *dz = O_S7[i][0]; *dy = O_S7[i][1]; *dx = O_S7[i][2]; return; }
  /* S13: all (dz,dy,dx) in {-1,0,1}^3 lexicographically before (0,0,0) */
  int t = 0;
  for (int a = -1; a <= 1; a++)
    for (int b = -1; b <= 1; b++)
      for (int cc = -1; cc <= 1; cc++) {
        if (a == 0 && b == 0 && cc == 0) return;
        if (t == i) { *dz = a; *dy = b; *dx = cc; return; }
        t++;
      }
}

/* Lorenzo weights over stencil k: the SZ formula (Section IV.A) with n = 1 in 3-D. */
static int o_lz_weight(int k, int i) {
  if (k == 7) return O_LZ7[i];
  int dz, dy, dx;
  o_stencil(k, i, &dz, &dy, &dx);
  if (dz > 0 || dy > 0 || dx > 0) return 0;
  int cnt = (dz != 0) + (dy != 0) + (dx != 0);
  return (cnt % 2 == 1) ? 1 : -1;
}

int orc_lz_weight(int k, int i) { return o_lz_weight(k, i); }

static int64_t o_lorenzo(const int32_t* v7) {
  int64_t s = 0;
  for (int i = 0; i < 7; i++) s += (int64_t)O_LZ7[i] * v7[i];
  return s;
}

/* Weight blob: W1[h1][k], b1[h1], (W2[h2][h1], b2[h2] if h2 > 0), W3[hl], b3. */
int orc_mlp_nweights(int k, int h1, int h2) {
  int hl = h2 > 0 ? h2 : h1;
  return h1 * k + h1 + (h2 > 0 ? h2 * h1 + h2 : 0) + hl + 1;
}

#define O_ALPHA 0.0625f /* leaky ReLU slope 2^-4 (Reading: slope unstated) */
#define O_MAXH 64

/* FP32 perceptron forward on centred integer inputs (Section IV.B, Fig. 3).
 * u_i = v_i 2^-s; each unit: acc = bias, then acc = fma(w, u_i, acc) in input
 * order; leaky ReLU on hidden units; linear output o; prediction o 2^s. */
float orc_mlp_fwd32(const float* w, int k, int h1, int h2, int s_in, const int32_t* v) {
  float sig = ldexpf(1.0f, -s_in);
  float u[32];
  for (int i = 0; i < k; i++) u[i] = (float)v[i] * sig;
  const float* W1 = w;
  const float* b1 = W1 + h1 * k;
  float a1[O_MAXH];
  for (int j = 0; j < h1; j++) {
    float acc = b1[j];
    for (int i = 0; i < k; i++) acc = fmaf(W1[j * k + i], u[i], acc);
    a1[j] = acc >= 0.0f ? acc : acc * O_ALPHA;
  }
  const float* p = b1 + h1;
  float* hl = a1;
  int nl = h1;
  float a2[O_MAXH];
  if (h2 > 0) {
    const float* W2 = p;
    const float* b2 = W2 + h2 * h1;
    for (int j = 0; j < h2; j++) {
      float acc = b2[j];
      for (int i = 0; i < h1; i++) acc = fmaf(W2[j * h1 + i], a1[i], acc);
      a2[j] = acc >= 0.0f ? acc : acc * O_ALPHA;
    }
    p = b2 + h2;
    hl = a2;
    nl = h2;
  }
  const float* W3 = p;
  float o = W3[nl];
  for (int j = 0; j < nl; j++) o = fmaf(W3[j], hl[j], o);
  return o * ldexpf(1.0f, s_in);
}

static int32_t o_round_pred(float p) {
  if (p != p) return 0;
  if (p > 1073741824.0f) p = 1073741824.0f;
  if (p < -1073741824.0f) p = -1073741824.0f;
  return (int32_t)rintf(p);
}

int32_t orc_mlp_pred32(const float* w, int k, int h1, int h2, int s_in, const int32_t* v) {
  return o_round_pred(orc_mlp_fwd32(w, k, h1, h2, s_in, v));
}

/* FP64 form of the same network (Section IV.B), for reporting only: the
 * FP32 weights taken exactly into double, u_i = v_i 2^-s, each unit
 * acc = bias, then acc = fma(w, u_i, acc) in input order, leaky ReLU slope
 * 2^-4, linear output, prediction rint(o 2^s) clamped to +-2^30.  Prediction
 * error and compression ratio are reported against this predictor; the
 * device never encodes with it. */
double orc_mlp_fwd64(const float* w, int k, int h1, int h2, int s_in, const int32_t* v) {
  double sig = ldexp(1.0, -s_in);
  double u[32];
  for (int i = 0; i < k; i++) u[i] = (double)v[i] * sig;
  const float* W1 = w;
  const float* b1 = W1 + h1 * k;
  double a1[O_MAXH];
  for (int j = 0; j < h1; j++) {
    double acc = (double)b1[j];
    for (int i = 0; i < k; i++) acc = fma((double)W1[j * k + i], u[i], acc);
    a1[j] = acc >= 0.0 ? acc : acc * (double)O_ALPHA;
  }
  const float* p = b1 + h1;
  double* hl = a1;
  int nl = h1;
  double a2[O_MAXH];
  if (h2 > 0) {
    const float* W2 = p;
    const float* b2 = W2 + h2 * h1;
    for (int j = 0; j < h2; j++) {
      double acc = (double)b2[j];
      for (int i = 0; i < h1; i++) acc = fma((double)W2[j * h1 + i], a1[i], acc);
      a2[j] = acc >= 0.0 ? acc : acc * (double)O_ALPHA;
    }
    p = b2 + h2;
    hl = a2;
    nl = h2;
  }
  const float* W3 = p;
  double o = (double)W3[nl];
  for (int j = 0; j < nl; j++) o = fma((double)W3[j], hl[j], o);
  return o * ldexp(1.0, s_in);
}

int32_t orc_mlp_pred64(const float* w, int k, int h1, int h2, int s_in, const int32_t* v) {
  double p = orc_mlp_fwd64(w, k, h1, h2, s_in, v);
  if (p != p) return 0;
  if (p > 1073741824.0) p = 1073741824.0;
  if (p < -1073741824.0) p = -1073741824.0;
  return (int32_t)rint(p);
}

/* ------------------------------------------------------------------------- */
/* Fixed-point (BF16) form of the perceptron (Section IV.B network, the      */
/* precision form evaluated on bf16 tensor-core operands).                    */
/*                                                                           */
/* Reading (the paper fixes no inference precision): every weight of layer l */
/* is an integer |Wq| <= 255 times 2^-e_l, so it is exactly a bf16 value;    */
/* the stencil inputs are the centred codes clamped to +-(2^16 - 1); the      */
/* hidden activations are integers clamped to +-(2^15 - 1).  Each layer's    */
/* sum of products is therefore an exact integer, computed here in int64.   */
/* (A tensor-core evaluation splits inputs and activations into 8-bit limbs, */
/* x = 256 hi + lo with 0 <= lo < 256, so each partial sum stays below 2^24  */
/* and FP32 accumulation is exact in any order and MMA shape.)  Per layer:   */
/*   A = sum Wq x + Bq;   leaky(A) = A >= 0 ? A : A / 16   (slope 2^-4)      */
/*   hidden:  Hq = clamp(rhu(leaky(A) 2^-t), +-(2^15 - 1)),  t >= 0          */
/*   output:  pred = clamp(rne(A 2^-F), +-2^30),  F = sum e - sum t          */
/* rhu = round half up, floor(y + 1/2); rne = round to nearest, ties to even.*/
/* Units: A_1 counts 2^-(e1 + s_in), so B1 = rint(b1 2^(e1 + s_in)); each    */
/* later layer's bias takes the units of its sum (orc_quantize); biases are  */
/* clamped to +-2^30, so every hidden sum fits 32 bits.                      */
/* qnet (int64): k, h1, h2, s_in, e1, e2, e3, t1, t2, then W1[h1][k], B1[h1], */
/* and for h2 > 0: W2[h2][h1], B2[h2], W3[h2], B3; for h2 = 0: W2[h1], B2    */
/* (e3 = t2 = 0).                                                             */
/* ------------------------------------------------------------------------- */
#define O_QHDR 9
#define O_QIN 65535
#define O_QH 32767

int orc_qnet_len(int k, int h1, int h2) {
  return O_QHDR + h1 * k + h1 + (h2 ? h2 * h1 + h2 + h2 + 1 : h1 + 1);
}

/* rne(x 2^-s) for integer x */
static int64_t o_rne_shift(int64_t x, int s) {
  if (s <= 0) return x * ((int64_t)1 << (-s));
  if (s >= 62) return 0;
  int64_t d = (int64_t)1 << s;
  int64_t q = x / d, r = x % d;
  if (r < 0) { q -= 1; r += d; }
  int64_t h = d >> 1;
  if (r > h || (r == h && (q & 1))) q += 1;
  return q;
}

/* floor(x 2^-s + 1/2) for integer x, s >= 0 */
static int64_t o_rhu_shift(int64_t x, int s) {
  if (s <= 0) return x;
  int64_t d = (int64_t)1 << s;
  int64_t y = x + (d >> 1);
  int64_t q = y / d;
  if (y % d != 0 && y < 0) q -= 1;  /* floor */
  return q;
}

static int64_t o_leaky_requant(int64_t a, int t) {
  int64_t h = a >= 0 ? o_rhu_shift(a, t) : o_rhu_shift(a, t + 4);
  return h > O_QH ? O_QH : (h < -O_QH ? -O_QH : h);
}

/* 16 |leaky(A)|: the activation magnitude that sets the shift t */
static int64_t o_leaky16(int64_t a) { return a >= 0 ? 16 * a : -a; }

/* hidden activations of layer 1 (and 2), writing the integer pre-activations */
static void o_q_hidden(const int64_t* q, const int32_t* v, int64_t* a1, int64_t* h1q, int64_t* a2, int64_t* h2q) {
  int k = (int)q[0], h1 = (int)q[1], h2 = (int)q[2];
  int t1 = (int)q[7], t2 = (int)q[8];
  const int64_t* W1 = q + O_QHDR;
  const int64_t* B1 = W1 + h1 * k;
  int64_t x[13];
  for (int i = 0; i < k; i++) x[i] = v[i] > O_QIN ? O_QIN : (v[i] < -O_QIN ? -O_QIN : v[i]);
  for (int j = 0; j < h1; j++) {
    int64_t acc = 0;
    for (int i = 0; i < k; i++) acc += W1[j * k + i] * x[i];
    a1[j] = acc + B1[j];
    h1q[j] = o_leaky_requant(a1[j], t1);
  }
  if (h2 && a2) {
    const int64_t* W2 = B1 + h1;
    const int64_t* B2 = W2 + h2 * h1;
    for (int j = 0; j < h2; j++) {
      int64_t acc = 0;
      for (int i = 0; i < h1; i++) acc += W2[j * h1 + i] * h1q[i];
      a2[j] = acc + B2[j];
      h2q[j] = o_leaky_requant(a2[j], t2);
    }
  }
}

int32_t orc_mlp_pred_q(const int64_t* q, const int32_t* v) {
  int k = (int)q[0], h1 = (int)q[1], h2 = (int)q[2];
  int e1 = (int)q[4], e2 = (int)q[5], e3 = (int)q[6], t1 = (int)q[7], t2 = (int)q[8];
  int64_t a1[O_MAXH], h1q[O_MAXH], a2[O_MAXH], h2q[O_MAXH];
  o_q_hidden(q, v, a1, h1q, a2, h2q);
  const int64_t* B1 = q + O_QHDR + h1 * k;
  int64_t acc;
  int F;
  if (h2) {
    const int64_t* W3 = B1 + h1 + h2 * h1 + h2;
    acc = W3[h2];
    int64_t s = 0;
    for (int j = 0; j < h2; j++) s += W3[j] * h2q[j];
    acc += s;
    F = e1 + e2 + e3 - t1 - t2;
  } else {
    const int64_t* W2 = B1 + h1;
    int64_t s = 0;
    for (int j = 0; j < h1; j++) s += W2[j] * h1q[j];
    acc = s + W2[h1];
    F = e1 + e2 - t1;
  }
  int64_t p = o_rne_shift(acc, F);
  if (p > 1073741824LL) p = 1073741824LL;
  if (p < -1073741824LL) p = -1073741824LL;
  return (int32_t)p;
}

/* Largest e with max|w| 2^e <= 255 (0 for all-zero weights), kept in [-30, 30]. */
static int o_wexp(const float* w, int n, int stride, int rows, int cols) {
  float m = 0.0f;
  for (int r = 0; r < rows; r++)
    for (int c = 0; c < cols; c++) {
      float a = fabsf(w[r * stride + c]);
      if (a > m) m = a;
    }
  (void)n;
  if (m == 0.0f) return 0;
  int E;
  float fr = frexpf(m, &E);
  int e = fr <= 255.0f / 256.0f ? 8 - E : 7 - E;
  return e < -30 ? -30 : (e > 30 ? 30 : e);
}

static int64_t o_qw(float w, int e) { return (int64_t)rintf(ldexpf(w, e)); }

static int64_t o_qb(float b, int E) {
  double v = rint(ldexp((double)b, E));
  const double lim = 1073741824.0; /* 2^30 */
  return (int64_t)(v > lim ? lim : (v < -lim ? -lim : v));
}

/* Smallest t in [0, 40] with M 2^-t <= 16 (2^15 - 1), M = max 16|leaky(A)|. */
static int o_shift_for(int64_t M) {
  const int64_t lim = 16 * (int64_t)O_QH;
  for (int t = 0; t < 40; t++)
    if (M <= (lim << t)) return t;
  return 40;
}

/* Quantize FP32 weights w (orc_mlp layout) with input scale s_in into qnet,
 * choosing the activation shifts from the used training and validation
 * samples (inputs tin/vin as gathered for training). */
int orc_qnet_build(const float* w, int k, int h1, int h2, int s_in, const int32_t* tin, const uint8_t* tus,
                   uint64_t nt, const int32_t* vin, const uint8_t* vus, uint64_t nv, int64_t* q) {
  int hl = h2 ? h2 : h1;
  const float* W1 = w;
  const float* b1 = W1 + h1 * k;
  const float* W2 = b1 + h1;
  const float* b2 = h2 ? W2 + h2 * h1 : NULL;
  const float* W3 = h2 ? b2 + h2 : W2;
  const float* b3 = W3 + hl;
  int e1 = o_wexp(W1, h1 * k, k, h1, k);
  int e2 = h2 ? o_wexp(W2, h2 * h1, h1, h2, h1) : o_wexp(W2, h1, h1, 1, h1);
  int e3 = h2 ? o_wexp(W3, h2, h2, 1, h2) : 0;
  q[0] = k; q[1] = h1; q[2] = h2; q[3] = s_in;
  q[4] = e1; q[5] = e2; q[6] = e3; q[7] = 0; q[8] = 0;
  int64_t* QW1 = q + O_QHDR;
  int64_t* QB1 = QW1 + h1 * k;
  for (int j = 0; j < h1 * k; j++) QW1[j] = o_qw(W1[j], e1);
  for (int j = 0; j < h1; j++) QB1[j] = o_qb(b1[j], e1 + s_in);
  int64_t* QW2 = QB1 + h1;
  int64_t* QB2 = h2 ? QW2 + h2 * h1 : QW2 + h1;
  int64_t* QW3 = h2 ? QB2 + h2 : NULL;
  int64_t* QB3 = h2 ? QW3 + h2 : NULL;
  /* layer-2 weights (integers) are needed for the layer-2 scan */
  if (h2) for (int j = 0; j < h2 * h1; j++) QW2[j] = o_qw(W2[j], e2);
  else for (int j = 0; j < h1; j++) QW2[j] = o_qw(W2[j], e2);
  int64_t a1[O_MAXH], h1q[O_MAXH], a2[O_MAXH], h2q[O_MAXH];
  /* t1 from the layer-1 pre-activations */
  int64_t M = 0;
  for (int pass = 0; pass < 2; pass++) {
    const int32_t* in = pass ? vin : tin;
    const uint8_t* us = pass ? vus : tus;
    uint64_t cnt = pass ? nv : nt;
    for (uint64_t s = 0; s < cnt; s++) {
      if (!us[s]) continue;
      o_q_hidden(q, in + s * (uint64_t)k, a1, h1q, NULL, NULL);
      for (int j = 0; j < h1; j++) if (o_leaky16(a1[j]) > M) M = o_leaky16(a1[j]);
    }
  }
  int t1 = o_shift_for(M);
  q[7] = t1;
  if (h2) {
    for (int j = 0; j < h2; j++) QB2[j] = o_qb(b2[j], e1 + e2 + s_in - t1);
    M = 0;
    for (int pass = 0; pass < 2; pass++) {
      const int32_t* in = pass ? vin : tin;
      const uint8_t* us = pass ? vus : tus;
      uint64_t cnt = pass ? nv : nt;
      for (uint64_t s = 0; s < cnt; s++) {
        if (!us[s]) continue;
        o_q_hidden(q, in + s * (uint64_t)k, a1, h1q, a2, h2q);
        for (int j = 0; j < h2; j++) if (o_leaky16(a2[j]) > M) M = o_leaky16(a2[j]);
      }
    }
    int t2 = o_shift_for(M);
    q[8] = t2;
    for (int j = 0; j < h2; j++) QW3[j] = o_qw(W3[j], e3);
    QB3[0] = o_qb(b3[0], e1 + e2 + e3 + s_in - t1 - t2);
  } else {
    QB2[0] = o_qb(b3[0], e1 + e2 + s_in - t1);
  }
  return ORC_OK;
}

static int o_bitlen(uint64_t n) { int b = 0; while (n) { b++; n >>= 1; } return b; }

/* ------------------------------------------------------------------------- */
/* Step a10: Huffman code lengths (Section IV.A stage 3; Section IV.C).      */
/* The code order handed to the canonical construction is the reverse of    */
/* the sorted leaf list (most frequent first), as an ordered symbol list in */
/* the style of ITU-T T.81 Annex C (BITS/HUFFVAL).                          */
/* Textbook Huffman: repeatedly join the two lightest nodes.  Total order:   */
/* (weight, leaf before internal node, leaves by symbol, internal nodes by   */
/* creation).  A single used symbol gets length 1.  Lengths are then handed   */
/* out by rank from the per-length counts: the lightest leaf gets the longest */
/* length.  If the longest exceeds lmax, the counts are first adjusted by the */
/* procedure of ITU-T T.81 Annex K.3 (move a deepest sibling pair up one      */
/* level and split a shallower leaf), which keeps the Kraft sum at one.       */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t f; uint32_t s; } o_leaf;
static int o_cmp_leaf(const void* a, const void* b) {
  const o_leaf* x = (const o_leaf*)a;
  const o_leaf* y = (const o_leaf*)b;
  if (x->f != y->f) return x->f < y->f ? -1 : 1;
  return x->s < y->s ? -1 : (x->s > y->s ? 1 : 0);
}

int orc_huffman_lengths(const uint64_t* hist, int nsym, int lmax, uint8_t* len, uint32_t* order) {
  memset(len, 0, (size_t)nsym);
  int n = 0;
  for (int s = 0; s < nsym; s++) n += hist[s] > 0;
  if (n == 0) return 0;
  o_leaf* L = (o_leaf*)malloc(sizeof(o_leaf) * (size_t)n);
  int t = 0;
  for (int s = 0; s < nsym; s++)
    if (hist[s] > 0) { L[t].f = hist[s]; L[t].s = (uint32_t)s; t++; }
  if (n == 1) { len[L[0].s] = 1; if (order) order[0] = L[0].s; free(L); return 1; }
  qsort(L, (size_t)n, sizeof(o_leaf), o_cmp_leaf);
  int nn = 2 * n - 1;
  uint64_t* w = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nn);
  int* parent = (int*)malloc(sizeof(int) * (size_t)nn);
  int* depth = (int*)malloc(sizeof(int) * (size_t)nn);
  for (int i = 0; i < n; i++) w[i] = L[i].f;
  int li = 0, ii = n, next = n;
  for (int step = 0; step < n - 1; step++) {
    int pick[2];
    for (int q = 0; q < 2; q++) {
      if (li < n && (ii >= next || w[li] <= w[ii])) pick[q] = li++;
      else pick[q] = ii++;
    }
    w[next] = w[pick[0]] + w[pick[1]];
    parent[pick[0]] = next;
    parent[pick[1]] = next;
    next++;
  }
  depth[nn - 1] = 0;
  for (int i = nn - 2; i >= 0; i--) depth[i] = depth[parent[i]] + 1;
  int maxlen = 0;
  int* bits = (int*)calloc((size_t)n + 2, sizeof(int));
  for (int i = 0; i < n; i++) { bits[depth[i]]++; if (depth[i] > maxlen) maxlen = depth[i]; }
  if (maxlen > lmax) {
    for (int i = maxlen; i > lmax; i--) {
      while (bits[i] > 0) {
        int j = i - 2;
        while (bits[j] == 0) j--;
        bits[i] -= 2;
        bits[i - 1] += 1;
        bits[j + 1] += 2;
        bits[j] -= 1;
      }
    }
    maxlen = lmax;
  }
  int idx = 0;
  for (int l = maxlen; l >= 1; l--)
    for (int c = 0; c < bits[l]; c++) len[L[idx++].s] = (uint8_t)l;
  if (order)
    for (int i = 0; i < n; i++) order[i] = L[n - 1 - i].s;
  free(bits); free(depth); free(parent); free(w); free(L);
  return n;
}

/* Canonical code words along a given symbol order whose lengths never
 * decrease: the first code is all zeros and each next code is the previous
 * plus one, shifted left by the growth in length.  This is the construction
 * of RFC 1951 Section 3.2.2 (there the order is by length, then symbol) and
 * of ITU-T T.81 Annex C (there the order is HUFFVAL). */
int orc_canonical_codes(const uint32_t* order, int n, const uint8_t* len, uint32_t* code) {
  uint32_t c = 0;
  int prev = 0;
  for (int i = 0; i < n; i++) {
    int l = len[order[i]];
    if (l < prev || l < 1) return ORC_ERR_ARG;
    if (i > 0) c = (c + 1u) << (l - prev);
    code[order[i]] = c;
    prev = l;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Container (little-endian).  Header of 256 bytes, then 16-byte aligned      */
/* sections: weights, codebook (sym | len << 16, by symbol), per-block bit    */
/* counts (| perceptron flag << 31), per-block balance-point counts (u16),   */
/* balance-point values (dtype), bitstream (u32 words, MSB first).           */
/* The factors travel with the stream (Section V).                           */
/* ------------------------------------------------------------------------- */
#define O_LMAX 24
#define O_HDR 256
static void put32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void put64(uint8_t* p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t get32(const uint8_t* p) { uint32_t v = 0; for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i); return v; }
static uint64_t get64(const uint8_t* p) { uint64_t v = 0; for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i); return v; }
static uint64_t al16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }

/* ------------------------------------------------------------------------- */
/* Section IV.A, the fourth SZ stage: a lossless pass over the bitstream      */
/* bytes (the paper names it; Algorithm 1 does not use it).  This build's     */
/* stage is an LZ77-style matcher over independent chunks of ORC_LZ_CHUNK    */
/* bytes, so that every chunk codes and decodes on its own:                  */
/*  - tokens: a control byte c < 128 is followed by c + 1 literal bytes; a   */
/*    control byte c >= 128 is a match of (c - 128) + 4 bytes (4..131) at a  */
/*    distance d (1..chunk) given by the next two bytes, little-endian;      */
/*  - greedy parse: at position i (with 4 bytes left) the hash of the 4      */
/*    bytes at i, h = (b0 | b1 << 8 | b2 << 16 | b3 << 24) * 2654435761 >>  */
/*    20 (Knuth's multiplicative hashing), names the last position that      */
/*    started a parse step with the same hash; if at least 4 bytes match     */
/*    there, the longest match up to 131 bytes is taken, else one literal;  */
/*    the table then names i; literals are emitted in runs of up to 128 just */
/*    before the next match or the chunk's end;                              */
/*  - a chunk whose tokens are not shorter than the chunk is stored as is.   */
/* Section: u32 chunk count, u32 chunk bytes, u64 raw bytes, then per chunk  */
/* u32 (coded bytes | stored << 31), 16-byte aligned, then the chunks'      */
/* bytes back to back.                                                        */
/* ------------------------------------------------------------------------- */
#define O_LZ_HB 12
static uint32_t o_lz_hash(const uint8_t* p) {
  uint32_t v = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
  return (v * 2654435761u) >> (32 - O_LZ_HB);
}

static size_t o_lz_lits(const uint8_t* src, size_t a, size_t b, uint8_t* dst, size_t o) {
  while (a < b) {
    size_t r = b - a < 128 ? b - a : 128;
    dst[o++] = (uint8_t)(r - 1);
    memcpy(dst + o, src + a, r);
    o += r;
    a += r;
  }
  return o;
}

/* tokens of one chunk (dst holds n + n / 128 + 1 bytes); returns their size */
static size_t o_lz_chunk(const uint8_t* src, size_t n, uint8_t* dst) {
  uint16_t tab[1 << O_LZ_HB];
  memset(tab, 0, sizeof(tab));
  size_t i = 0, lit0 = 0, o = 0;
  while (i < n) {
    size_t L = 0, d = 0;
    if (i + 4 <= n) {
      uint32_t h = o_lz_hash(src + i);
      size_t cand = tab[h];
      tab[h] = (uint16_t)(i + 1);
      if (cand) {
        size_t j = cand - 1;
        while (i + L < n && L < 131 && src[j + L] == src[i + L]) L++;
        if (L >= 4) d = i - j;
        else L = 0;
      }
    }
    if (L) {
      o = o_lz_lits(src, lit0, i, dst, o);
      dst[o++] = (uint8_t)(128 + (L - 4));
      dst[o++] = (uint8_t)(d & 0xFF);
      dst[o++] = (uint8_t)(d >> 8);
      i += L;
      lit0 = i;
    } else {
      i++;
    }
  }
  return o_lz_lits(src, lit0, n, dst, o);
}

uint64_t orc_lz_bound(uint64_t raw) {
  uint64_t nch = (raw + ORC_LZ_CHUNK - 1) / ORC_LZ_CHUNK;
  return al16(16 + 4 * nch) + raw + 16;
}

uint64_t orc_lz_encode(const uint8_t* src, uint64_t raw, uint8_t* out) {
  uint64_t nch = (raw + ORC_LZ_CHUNK - 1) / ORC_LZ_CHUNK;
  put32(out, (uint32_t)nch);
  put32(out + 4, ORC_LZ_CHUNK);
  put64(out + 8, raw);
  uint64_t o = al16(16 + 4 * nch);
  memset(out + 16, 0, o - 16);
  uint8_t* tmp = (uint8_t*)malloc(ORC_LZ_CHUNK + ORC_LZ_CHUNK / 128 + 8);
  for (uint64_t c = 0; c < nch; c++) {
    uint64_t a = c * ORC_LZ_CHUNK;
    size_t n = (size_t)(raw - a < ORC_LZ_CHUNK ? raw - a : ORC_LZ_CHUNK);
    size_t sz = o_lz_chunk(src + a, n, tmp);
    if (sz >= n) {
      memcpy(out + o, src + a, n);
      put32(out + 16 + 4 * c, (uint32_t)n | 0x80000000u);
      o += n;
    } else {
      memcpy(out + o, tmp, sz);
      put32(out + 16 + 4 * c, (uint32_t)sz);
      o += sz;
    }
  }
  free(tmp);
  return o;
}

/* Decode a section of sec_bytes into raw bytes; ORC_ERR_CORRUPT on any
 * inconsistency (sizes, token bounds, distances). */
int orc_lz_decode(const uint8_t* sec, uint64_t sec_bytes, uint8_t* dst, uint64_t raw) {
  if (sec_bytes < 16) return ORC_ERR_CORRUPT;
  uint64_t nch = get32(sec), chunk = get32(sec + 4), r = get64(sec + 8);
  if (chunk != ORC_LZ_CHUNK || r != raw || nch != (raw + ORC_LZ_CHUNK - 1) / ORC_LZ_CHUNK) return ORC_ERR_CORRUPT;
  uint64_t o = al16(16 + 4 * nch);
  if (o > sec_bytes) return ORC_ERR_CORRUPT;
  for (uint64_t c = 0; c < nch; c++) {
    uint32_t e = get32(sec + 16 + 4 * c);
    uint64_t sz = e & 0x7FFFFFFFu, a = c * ORC_LZ_CHUNK;
    uint64_t n = raw - a < ORC_LZ_CHUNK ? raw - a : ORC_LZ_CHUNK;
    if (o + sz > sec_bytes) return ORC_ERR_CORRUPT;
    const uint8_t* t = sec + o;
    uint8_t* d = dst + a;
    if (e >> 31) {
      if (sz != n) return ORC_ERR_CORRUPT;
      memcpy(d, t, n);
    } else {
      uint64_t p = 0, q = 0;
      while (p < sz) {
        uint32_t cb = t[p++];
        if (cb < 128) {
          uint64_t L = cb + 1;
          if (p + L > sz || q + L > n) return ORC_ERR_CORRUPT;
          memcpy(d + q, t + p, L);
          p += L;
          q += L;
        } else {
          uint64_t L = cb - 128 + 4;
          if (p + 2 > sz) return ORC_ERR_CORRUPT;
          uint64_t dist = (uint64_t)t[p] | ((uint64_t)t[p + 1] << 8);
          p += 2;
          if (dist < 1 || dist > q || q + L > n) return ORC_ERR_CORRUPT;
          for (uint64_t k = 0; k < L; k++, q++) d[q] = d[q - dist];
        }
      }
      if (q != n) return ORC_ERR_CORRUPT;
    }
    o += sz;
  }
  return o == sec_bytes ? ORC_OK : ORC_ERR_CORRUPT;
}

typedef struct {
  uint64_t nb[3], nblocks, bvol;
} o_geom;

static int o_geom_make(const uint64_t dims[3], const int block[3], o_geom* g) {
  uint64_t vol = 1;
  for (int i = 0; i < 3; i++) {
    if (block[i] < 1 || dims[i] < 1) return ORC_ERR_ARG;
    g->nb[i] = (dims[i] + (uint64_t)block[i] - 1) / (uint64_t)block[i];
    vol *= (uint64_t)block[i];
  }
  if (vol > 4096 || vol < 2) return ORC_ERR_ARG;
  g->bvol = vol;
  g->nblocks = g->nb[0] * g->nb[1] * g->nb[2];
  return ORC_OK;
}

uint64_t orc_compress_bound(const uint64_t dims[3], int dtype, const int block[3], int m, int nweights) {
  o_geom g;
  if (o_geom_make(dims, block, &g)) return 0;
  uint64_t n = dims[0] * dims[1] * dims[2];
  uint64_t ts = dtype == ORC_F64 ? 8 : 4;
  uint64_t b = O_HDR;
  b = al16(b + 4ull * (uint64_t)nweights);
  b = al16(b + 4ull * (1ull << m));
  b = al16(b + 4ull * g.nblocks);
  b = al16(b + 2ull * g.nblocks);
  b = al16(b + ts * n);
  b = al16(b + 4ull * ((n * O_LMAX + 31) / 32 + 1));
  /* the lossless stage's chunk table (a stored chunk is never longer than itself) */
  b += orc_lz_bound(4ull * ((n * O_LMAX + 31) / 32 + 1)) - 4ull * ((n * O_LMAX + 31) / 32 + 1);
  return b;
}

/* a5-a8 of one block (Section IV.A, IV.B, IV.D; Alg. 1): dqb[j], okb[j] are
 * the codes and bound flags of the block's points in local raster order
 * (e0 x e1 x e2, truncated at the field's edge).  Centres the codes on the
 * anchor (j = 0), predicts every other point by Lorenzo and, if use_nn, by
 * the perceptron from its causal in-block neighbours, quantizes both into
 * cz / cn (code k + R, or 0 for a balance point), and returns 1 when the
 * perceptron's residual bits are strictly fewer (the block then uses cn). */
static int o_block(const int32_t* dqb, const uint8_t* okb, int e0, int e1, int e2, const orc_params* p, int use_nn,
                   int use_q, int use_64, int k, int64_t R, int32_t* vc, int64_t* vt, uint16_t* cz, uint16_t* cn) {
  int32_t da = dqb[0];
  for (int j = 0; j < e0 * e1 * e2; j++) {
    int64_t v = (int64_t)dqb[j] - (int64_t)da;
    vt[j] = v;
    vc[j] = (int32_t)(v > O_VCLAMP ? O_VCLAMP : (v < -O_VCLAMP ? -O_VCLAMP : v));
  }
  int64_t costz = 0, costn = 0;
  for (int lz = 0; lz < e0; lz++)
    for (int ly = 0; ly < e1; ly++)
      for (int lx = 0; lx < e2; lx++) {
        int j = (lz * e1 + ly) * e2 + lx;
        if (j == 0) continue;
        int32_t in7[7];
        for (int i = 0; i < 7; i++) {
          int qz = lz + O_S7[i][0], qy = ly + O_S7[i][1], qx = lx + O_S7[i][2];
          in7[i] = (qz >= 0 && qy >= 0 && qx >= 0) ? vc[(qz * e1 + qy) * e2 + qx] : 0;
        }
        int64_t kz = vt[j] - o_lorenzo(in7);
        int64_t az = kz < 0 ? -kz : kz;
        costz += o_bitlen((uint64_t)(az < R ? az : R));
        cz[j] = (uint16_t)((az <= R - 1 && okb[j]) ? kz + R : 0);
        if (use_nn) {
          int32_t in[13];
          for (int i = 0; i < k; i++) {
            int dz, dy, dx;
            o_stencil(k, i, &dz, &dy, &dx);
            int qz = lz + dz, qy = ly + dy, qx = lx + dx;
            in[i] = (qz >= 0 && qy >= 0 && qx >= 0 && qz < e0 && qy < e1 && qx < e2) ? vc[(qz * e1 + qy) * e2 + qx]
                                                                                      : 0;
          }
          int64_t pr = use_q ? (int64_t)orc_mlp_pred_q(p->qnet, in)
                       : use_64 ? (int64_t)orc_mlp_pred64(p->weights, k, p->h1, p->h2, p->s_in, in)
                                : (int64_t)orc_mlp_pred32(p->weights, k, p->h1, p->h2, p->s_in, in);
          int64_t kn = vt[j] - pr;
          int64_t an = kn < 0 ? -kn : kn;
          costn += o_bitlen((uint64_t)(an < R ? an : R));
          cn[j] = (uint16_t)((an <= R - 1 && okb[j]) ? kn + R : 0);
        }
      }
  /* a7: perceptron only where it is strictly cheaper than Lorenzo */
  return use_nn && costn < costz;
}

/* ------------------------------------------------------------------------- */
/* The paper-literal data selection (Section IV.D, float32 only): every      */
/* point is predicted from the true values of its causal in-block            */
/* neighbours, not from values the decoder can reproduce, so decompression,  */
/* which can only predict from its own reconstructions, drifts; balance      */
/* points (stored values, "equilibrium points") stop the drift.  Readings:   */
/*  - a value's real code is (t, K): t = L32(|x|) * inv in steps and K the  */
/*    factor offset of its sign class, for non-zero values that pass the     */
/*    bound check of the bound-safe transform; any other value (zero,        */
/*    subnormal, a failed check) has t = 0 and K = its integer code and is   */
/*    always stored as a balance point;                                      */
/*  - values enter the predictor centred on the block anchor:               */
/*    c = (t - t_a) + (K - K_a), clamped to +-(2^24 - 1);                   */
/*  - Lorenzo sums w_i c_i in stencil order; the FP32 perceptron takes       */
/*    u_i = c_i 2^-s and returns o 2^s, as for integer inputs;              */
/*  - residual k = rint(c - pred); the code is k + R when |k| <= R - 1,     */
/*    else 0 (balance point); with eq_period > 0, every eq_period-th point  */
/*    of the block in raster order is a deliberate balance point;           */
/*  - every block uses the given predictor (no per-block Lorenzo choice);   */
/*  - decoding walks each block serially in raster order: c' = pred(c'_nb)  */
/*    + k, z = c' + t_a, q' = rint(z) + K_a, and the value is 0 in the zero  */
/*    class, else the sign of the class times E32((z + K_a - K_cls) step).   */
/* ------------------------------------------------------------------------- */
static void o_realcode32(float x, const orc_consts* c, float* t, int64_t* K) {
  int32_t q;
  int ok;
  orc_transform32(x, c, &q, &ok);
  if (x != 0.0f && ok) {
    *t = orc_L32(fabsf(x)) * c->inv32;
    *K = x > 0.0f ? c->Kp : c->Kn;
  } else {
    *t = 0.0f;
    *K = q;
  }
}

static int o_lit_codable(float x, const orc_consts* c) {
  int32_t q;
  int ok;
  orc_transform32(x, c, &q, &ok);
  return x != 0.0f && ok;
}

static float o_cen(float t, int64_t K, float ta, int64_t Ka) { return (t - ta) + (float)(K - Ka); }

static float o_clampf(float v) { return v > 16777215.0f ? 16777215.0f : (v < -16777215.0f ? -16777215.0f : v); }

/* FP32 perceptron on real centred inputs: the arithmetic of orc_mlp_fwd32
 * with u_i = v_i 2^-s. */
static float o_mlp_fwd32f(const float* w, int k, int h1, int h2, int s_in, const float* v) {
  float sig = ldexpf(1.0f, -s_in);
  float u[32];
  for (int i = 0; i < k; i++) u[i] = v[i] * sig;
  const float* W1 = w;
  const float* b1 = W1 + h1 * k;
  float a1[O_MAXH];
  for (int j = 0; j < h1; j++) {
    float acc = b1[j];
    for (int i = 0; i < k; i++) acc = fmaf(W1[j * k + i], u[i], acc);
    a1[j] = acc >= 0.0f ? acc : acc * O_ALPHA;
  }
  const float* p = b1 + h1;
  float* hl = a1;
  int nl = h1;
  float a2[O_MAXH];
  if (h2 > 0) {
    const float* W2 = p;
    const float* b2 = W2 + h2 * h1;
    for (int j = 0; j < h2; j++) {
      float acc = b2[j];
      for (int i = 0; i < h1; i++) acc = fmaf(W2[j * h1 + i], a1[i], acc);
      a2[j] = acc >= 0.0f ? acc : acc * O_ALPHA;
    }
    p = b2 + h2;
    hl = a2;
    nl = h2;
  }
  const float* W3 = p;
  float o = W3[nl];
  for (int j = 0; j < nl; j++) o = fmaf(W3[j], hl[j], o);
  return o * ldexpf(1.0f, s_in);
}

/* The prediction of point (lz, ly, lx) of an e0 x e1 x e2 block from the
 * centred real values cv (raster order) of its causal in-block neighbours. */
static float o_lit_pred(const float* cv, int lz, int ly, int lx, int e0, int e1, int e2, const float* w, int k, int h1,
                        int h2, int s_in) {
  if (w) {
    float in[13];
    for (int i = 0; i < k; i++) {
      int dz, dy, dx;
      o_stencil(k, i, &dz, &dy, &dx);
      int qz = lz + dz, qy = ly + dy, qx = lx + dx;
      in[i] = (qz >= 0 && qy >= 0 && qx >= 0 && qz < e0 && qy < e1 && qx < e2) ? cv[(qz * e1 + qy) * e2 + qx] : 0.0f;
    }
    return o_mlp_fwd32f(w, k, h1, h2, s_in, in);
  }
  float acc = 0.0f;
  for (int i = 0; i < 7; i++) {
    int qz = lz + O_S7[i][0], qy = ly + O_S7[i][1], qx = lx + O_S7[i][2];
    float v = (qz >= 0 && qy >= 0 && qx >= 0) ? cv[(qz * e1 + qy) * e2 + qx] : 0.0f;
    acc = acc + (float)O_LZ7[i] * v;
  }
  return acc;
}

static int64_t o_lit_round(float r) {
  if (r != r) return 0;
  if (r > 1073741824.0f) r = 1073741824.0f;
  if (r < -1073741824.0f) r = -1073741824.0f;
  return (int64_t)rintf(r);
}

/* Codes of one block under the literal selection: x in raster order. */
static void o_block_literal(const float* xb, int e0, int e1, int e2, const orc_consts* c, const float* w, int k, int h1,
                            int h2, int s_in, int64_t R, int eq_period, float* cv, uint16_t* cs) {
  int np = e0 * e1 * e2;
  float ta;
  int64_t Ka;
  o_realcode32(xb[0], c, &ta, &Ka);
  for (int j = 0; j < np; j++) {
    float t;
    int64_t K;
    o_realcode32(xb[j], c, &t, &K);
    cv[j] = o_clampf(o_cen(t, K, ta, Ka));
  }
  for (int lz = 0; lz < e0; lz++)
    for (int ly = 0; ly < e1; ly++)
      for (int lx = 0; lx < e2; lx++) {
        int j = (lz * e1 + ly) * e2 + lx;
        if (j == 0) continue;
        if (!o_lit_codable(xb[j], c) || (eq_period > 0 && j % eq_period == 0)) { cs[j] = 0; continue; }
        float pr = o_lit_pred(cv, lz, ly, lx, e0, e1, e2, w, k, h1, h2, s_in);
        int64_t kk = o_lit_round(cv[j] - pr);
        int64_t a = kk < 0 ? -kk : kk;
        cs[j] = (uint16_t)(a <= R - 1 ? kk + R : 0);
      }
}

/* The literal decoder's value of a centred real code cc (anchor (ta, Ka)). */
static float o_lit_value(float cc, float ta, int64_t Ka, const orc_consts* c) {
  float z = cc + ta;
  int64_t q = o_lit_round(z) + Ka;
  if (q > 2147483647LL) q = 2147483647LL;
  if (q < -2147483647LL) q = -2147483647LL;
  int cl = o_class((int32_t)q, c);
  if (cl == 0) return 0.0f;
  int64_t Kc = cl == 1 ? c->Kp : c->Kn;
  float nr = z + (float)(Ka - Kc);
  float a = orc_E32(nr * c->step32);
  return cl == 1 ? a : -a;
}

/* A given codebook (sym | len << 16 per entry, in the order the container
 * stores it): symbols below 2^m and distinct, lengths 1..24 and never
 * decreasing along the list (the canonical construction needs that order),
 * Kraft sum at most one, and symbol 0 present, because balance points are
 * coded as symbol 0.  Fills lens (zero for symbols not in the list) and the
 * symbol order.  A single entry gets length 1, as the Huffman construction
 * gives a single used symbol. */
static int o_codebook_check(const uint32_t* cb, int n, int m, uint8_t* lens, uint32_t* order) {
  int nsym = 1 << m;
  if (n < 1 || n > nsym) return ORC_ERR_ARG;
  memset(lens, 0, (size_t)nsym);
  double kraft = 0.0;
  int prev = 1, have0 = 0;
  for (int t = 0; t < n; t++) {
    uint32_t sym = cb[t] & 0xFFFFu, l = cb[t] >> 16;
    if (sym >= (uint32_t)nsym || l < 1 || l > O_LMAX || (int)l < prev || lens[sym]) return ORC_ERR_ARG;
    if (n == 1 && l != 1) return ORC_ERR_ARG;
    lens[sym] = (uint8_t)l;
    order[t] = sym;
    prev = (int)l;
    kraft += ldexp(1.0, -(int)l);
    have0 |= sym == 0;
  }
  if (kraft > 1.0 || !have0) return ORC_ERR_ARG;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: compression.                                                  */
/* With p->codebook (Section IV.C: the Huffman code built in the training     */
/* phase from the validation set's averaged per-block code frequencies and    */
/* kept for the compression phase), the code words come from that list        */
/* instead of the field's own histogram, and a code the list does not hold    */
/* becomes a balance point (code 0, value stored) like any code outside the   */
/* quantization range.  The container then carries the list as its codebook   */
/* and places the bitstream before the balance-point values (header flag      */
/* ORC_FLAG_STREAM_FIRST), the order in which a single pass can write them.   */
/* ------------------------------------------------------------------------- */
int orc_compress(const void* x, const uint64_t dims[3], int dtype, const orc_params* p,
                 uint8_t* out, uint64_t cap, uint64_t* out_size, orc_dump* dump) {
  if (dtype != ORC_F32 && dtype != ORC_F64) return ORC_ERR_DTYPE;
  if (p->m < 2 || p->m > 16) return ORC_ERR_ARG;
  int use_q = p->pred == ORC_PRED_MLP_BF16 && p->qnet != NULL;
  int use_64 = p->pred == ORC_PRED_MLP64 && p->weights != NULL;
  int use_nn = ((p->pred == ORC_PRED_MLP || use_64) && p->weights != NULL) || use_q;
  int k = p->stencil;
  if (use_q && (p->qnet[0] != k || p->qnet[1] != p->h1 || p->qnet[2] != p->h2 || p->qnet[3] != p->s_in))
    return ORC_ERR_ARG;
  if (use_nn && (k != 7 && k != 13)) return ORC_ERR_ARG;
  if (use_nn && (p->h1 < 1 || p->h1 > O_MAXH || p->h2 < 0 || p->h2 > O_MAXH)) return ORC_ERR_ARG;
  if (use_nn && (p->s_in < 0 || p->s_in > 30)) return ORC_ERR_ARG;
  int lit = p->literal != 0;
  if (lit && (dtype != ORC_F32 || use_q || use_64 || p->codebook || p->eq_period < 0)) return ORC_ERR_ARG;
  if (p->lossless && p->codebook) return ORC_ERR_ARG;  /* the stage follows a stream that ends the container */
  o_geom g;
  if (o_geom_make(dims, p->block, &g)) return ORC_ERR_ARG;
  uint64_t n = dims[0] * dims[1] * dims[2];
  size_t ts = dtype == ORC_F64 ? 8 : 4;
  int nsym = 1 << p->m;
  int64_t R = (int64_t)1 << (p->m - 1);

  /* a1, a2 */
  double amin, amax;
  int trivial;
  int st = orc_stats(x, n, dtype, &amin, &amax, &trivial);
  if (st) return st;
  orc_consts c;
  st = orc_make_consts(dtype, amin, amax, trivial, p->eb, &c);
  if (st) return st;

  /* a4: transform every point (Alg. 1, the per-point map) */
  int32_t* dq = (int32_t*)malloc(sizeof(int32_t) * n);
  uint8_t* okv = (uint8_t*)malloc(n);
  for (uint64_t i = 0; i < n; i++) {
    int ok;
    if (dtype == ORC_F32) orc_transform32(((const float*)x)[i], &c, &dq[i], &ok);
    else orc_transform64(((const double*)x)[i], &c, &dq[i], &ok);
    okv[i] = (uint8_t)ok;
  }

  /* a given codebook: its lengths and symbol order */
  int fixed_cb = p->codebook != NULL;
  uint8_t* lens = (uint8_t*)malloc((size_t)nsym);
  uint32_t* cw = (uint32_t*)calloc((size_t)nsym, sizeof(uint32_t));
  uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nsym);
  if (fixed_cb && o_codebook_check(p->codebook, p->codebook_n, p->m, lens, order)) {
    free(lens); free(cw); free(order); free(dq); free(okv);
    return ORC_ERR_ARG;
  }

  /* a5-a9: per block predict, select, quantize, histogram */
  uint16_t* codes = (uint16_t*)calloc(g.nblocks * g.bvol, sizeof(uint16_t));
  uint8_t* nnf = (uint8_t*)calloc(g.nblocks, 1);
  uint16_t* nout = (uint16_t*)calloc(g.nblocks, sizeof(uint16_t));
  uint64_t* hist = (uint64_t*)calloc((size_t)nsym, sizeof(uint64_t));
  int32_t* vc = (int32_t*)malloc(sizeof(int32_t) * g.bvol);
  int64_t* vt = (int64_t*)malloc(sizeof(int64_t) * g.bvol);
  uint16_t* cz = (uint16_t*)malloc(sizeof(uint16_t) * g.bvol);
  uint16_t* cn = (uint16_t*)malloc(sizeof(uint16_t) * g.bvol);
  int32_t* dqb = (int32_t*)malloc(sizeof(int32_t) * g.bvol);
  uint8_t* okb = (uint8_t*)malloc(g.bvol);
  uint64_t n_out = 0;
  uint64_t bi = 0;
  for (uint64_t bz = 0; bz < g.nb[0]; bz++)
    for (uint64_t by = 0; by < g.nb[1]; by++)
      for (uint64_t bx = 0; bx < g.nb[2]; bx++, bi++) {
        uint64_t o0 = bz * p->block[0], o1 = by * p->block[1], o2 = bx * p->block[2];
        int e0 = (int)((dims[0] - o0) < (uint64_t)p->block[0] ? dims[0] - o0 : (uint64_t)p->block[0]);
        int e1 = (int)((dims[1] - o1) < (uint64_t)p->block[1] ? dims[1] - o1 : (uint64_t)p->block[1]);
        int e2 = (int)((dims[2] - o2) < (uint64_t)p->block[2] ? dims[2] - o2 : (uint64_t)p->block[2]);
        int np = e0 * e1 * e2;
        for (int lz = 0; lz < e0; lz++)
          for (int ly = 0; ly < e1; ly++)
            for (int lx = 0; lx < e2; lx++) {
              int j = (lz * e1 + ly) * e2 + lx;
              uint64_t ig = ((o0 + lz) * dims[1] + (o1 + ly)) * dims[2] + (o2 + lx);
              dqb[j] = dq[ig];
              okb[j] = okv[ig];
            }
        int usen;
        if (lit) {
          float* xb = (float*)malloc(sizeof(float) * (size_t)np);
          float* cvf = (float*)malloc(sizeof(float) * (size_t)np);
          for (int lz = 0; lz < e0; lz++)
            for (int ly = 0; ly < e1; ly++)
              for (int lx = 0; lx < e2; lx++)
                xb[(lz * e1 + ly) * e2 + lx] = ((const float*)x)[((o0 + lz) * dims[1] + (o1 + ly)) * dims[2] + (o2 + lx)];
          o_block_literal(xb, e0, e1, e2, &c, use_nn ? p->weights : NULL, k, p->h1, p->h2, p->s_in, R, p->eq_period,
                          cvf, cn);
          free(cvf);
          free(xb);
          usen = use_nn;
        } else {
          usen = o_block(dqb, okb, e0, e1, e2, p, use_nn, use_q, use_64, k, R, vc, vt, cz, cn);
        }
        nnf[bi] = (uint8_t)usen;
        const uint16_t* cs = (usen || lit) ? cn : cz;
        int no = 1;  /* the anchor */
        for (int j = 1; j < np; j++) {
          /* a code outside a given codebook is stored as a balance point */
          uint16_t cd = (fixed_cb && lens[cs[j]] == 0) ? 0 : cs[j];
          codes[bi * g.bvol + j] = cd;
          hist[cd]++;
          if (cd == 0) no++;
        }
        nout[bi] = (uint16_t)no;
        n_out += (uint64_t)no;
      }

  /* a10: code lengths and canonical codes (of the field's histogram, or the given list) */
  int n_used = fixed_cb ? p->codebook_n : orc_huffman_lengths(hist, nsym, O_LMAX, lens, order);
  orc_canonical_codes(order, n_used, lens, cw);

  /* a11: per-block bit counts and total */
  uint32_t* bbits = (uint32_t*)malloc(sizeof(uint32_t) * g.nblocks);
  uint64_t tbits = 0;
  bi = 0;
  for (uint64_t b = 0; b < g.nblocks; b++) {
    uint64_t bz = b / (g.nb[1] * g.nb[2]), by = (b / g.nb[2]) % g.nb[1], bx = b % g.nb[2];
    int e0 = (int)((dims[0] - bz * p->block[0]) < (uint64_t)p->block[0] ? dims[0] - bz * p->block[0] : (uint64_t)p->block[0]);
    int e1 = (int)((dims[1] - by * p->block[1]) < (uint64_t)p->block[1] ? dims[1] - by * p->block[1] : (uint64_t)p->block[1]);
    int e2 = (int)((dims[2] - bx * p->block[2]) < (uint64_t)p->block[2] ? dims[2] - bx * p->block[2] : (uint64_t)p->block[2]);
    int np = e0 * e1 * e2;
    uint32_t s = 0;
    for (int j = 1; j < np; j++) s += lens[codes[b * g.bvol + j]];
    bbits[b] = s;
    tbits += s;
  }
  uint64_t swords = (tbits + 31) / 32;

  /* layout */
  /* weights section: FP32 blob, or the int64 fixed-point network */
  int nw = use_q ? orc_qnet_len(k, p->h1, p->h2) : (use_nn ? orc_mlp_nweights(k, p->h1, p->h2) : 0);
  uint64_t off_w = O_HDR;
  uint64_t off_cb = al16(off_w + (use_q ? 8ull : 4ull) * (uint64_t)nw);
  uint64_t off_bb = al16(off_cb + 4ull * (uint64_t)n_used);
  uint64_t off_bn = al16(off_bb + 4ull * g.nblocks);
  uint64_t off_ov, off_st, total;
  if (fixed_cb) {
    off_st = al16(off_bn + 2ull * g.nblocks);
    off_ov = al16(off_st + 4ull * swords);
    total = al16(off_ov + ts * n_out);
  } else {
    off_ov = al16(off_bn + 2ull * g.nblocks);
    off_st = al16(off_ov + ts * n_out);
    total = al16(off_st + 4ull * swords);
  }
  int ret = ORC_OK;
  if (total > cap) { ret = ORC_ERR_CAPACITY; goto done; }
  memset(out, 0, total);

  /* header */
  memcpy(out, "PCMP", 4);
  put32(out + 4, 1);
  put32(out + 8, (uint32_t)dtype);
  put32(out + 12, (uint32_t)(use_q ? ORC_PRED_MLP_BF16 : (use_64 ? ORC_PRED_MLP64 : (use_nn ? ORC_PRED_MLP : ORC_PRED_LORENZO))));
  put64(out + 16, dims[0]); put64(out + 24, dims[1]); put64(out + 32, dims[2]);
  put32(out + 40, (uint32_t)p->block[0]); put32(out + 44, (uint32_t)p->block[1]); put32(out + 48, (uint32_t)p->block[2]);
  put32(out + 52, (uint32_t)(use_nn ? k : 0));
  put32(out + 56, (uint32_t)(use_nn ? p->h1 : 0));
  put32(out + 60, (uint32_t)(use_nn ? p->h2 : 0));
  put32(out + 64, (uint32_t)p->m);
  put32(out + 68, (uint32_t)(use_nn ? p->s_in : 0));
  put64(out + 72, bits_of_d(p->eb));
  put64(out + 80, bits_of_d(amin));
  put64(out + 88, bits_of_d(amax));
  put32(out + 96, (uint32_t)(trivial ? 1 : 0));
  put32(out + 100, (uint32_t)c.Kp); put32(out + 104, (uint32_t)c.Kn);
  put32(out + 108, (uint32_t)c.Zq); put32(out + 112, (uint32_t)c.S);
  put32(out + 116, (uint32_t)n_used);
  if (dtype == ORC_F32) {
    put64(out + 120, bits_of_f(c.step32)); put64(out + 128, bits_of_f(c.inv32)); put64(out + 136, bits_of_f(c.ebdn32));
  } else {
    put64(out + 120, bits_of_d(c.stepd)); put64(out + 128, bits_of_d(c.invd)); put64(out + 136, bits_of_d(c.ebdnd));
  }
  put64(out + 144, g.nblocks);
  put64(out + 152, n_out);
  put64(out + 160, swords);
  put64(out + 168, off_w); put64(out + 176, off_cb); put64(out + 184, off_bb);
  put64(out + 192, off_bn); put64(out + 200, off_ov); put64(out + 208, off_st);
  put64(out + 216, total);
  put32(out + 224, (uint32_t)nw);
  put32(out + 228, (fixed_cb ? ORC_FLAG_STREAM_FIRST : 0u) | (lit ? ORC_FLAG_LITERAL : 0u));
  put32(out + 232, lit ? (uint32_t)p->eq_period : 0u);
  put32(out + 252, orc_crc32(out, 252));

  /* sections */
  if (use_q) for (int i = 0; i < nw; i++) put64(out + off_w + 8ull * i, (uint64_t)p->qnet[i]);
  else for (int i = 0; i < nw; i++) put32(out + off_w + 4ull * i, bits_of_f(p->weights[i]));
  for (int t = 0; t < n_used; t++)
    put32(out + off_cb + 4ull * (uint64_t)t, order[t] | ((uint32_t)lens[order[t]] << 16));
  for (uint64_t b = 0; b < g.nblocks; b++) {
    put32(out + off_bb + 4ull * b, bbits[b] | ((uint32_t)nnf[b] << 31));
    out[off_bn + 2ull * b] = (uint8_t)(nout[b] & 0xFF);
    out[off_bn + 2ull * b + 1] = (uint8_t)(nout[b] >> 8);
  }
  {
    /* a12: balance points (anchor first, then code-0 points in raster order) and bits */
    uint64_t oi = 0, bp = 0;
    for (uint64_t b = 0; b < g.nblocks; b++) {
      uint64_t bz = b / (g.nb[1] * g.nb[2]), by = (b / g.nb[2]) % g.nb[1], bx = b % g.nb[2];
      uint64_t o0 = bz * p->block[0], o1 = by * p->block[1], o2 = bx * p->block[2];
      int e0 = (int)((dims[0] - o0) < (uint64_t)p->block[0] ? dims[0] - o0 : (uint64_t)p->block[0]);
      int e1 = (int)((dims[1] - o1) < (uint64_t)p->block[1] ? dims[1] - o1 : (uint64_t)p->block[1]);
      int e2 = (int)((dims[2] - o2) < (uint64_t)p->block[2] ? dims[2] - o2 : (uint64_t)p->block[2]);
      for (int lz = 0; lz < e0; lz++)
        for (int ly = 0; ly < e1; ly++)
          for (int lx = 0; lx < e2; lx++) {
            int j = (lz * e1 + ly) * e2 + lx;
            uint64_t ig = ((o0 + lz) * dims[1] + (o1 + ly)) * dims[2] + (o2 + lx);
            uint16_t cd = codes[b * g.bvol + j];
            if (j == 0 || cd == 0) {
              memcpy(out + off_ov + ts * oi, (const uint8_t*)x + ts * ig, ts);
              oi++;
            }
            if (j == 0) continue;
            uint32_t w = cw[cd];
            int L = lens[cd];
            for (int q = L - 1; q >= 0; q--, bp++) {
              if ((w >> q) & 1u) {
                uint64_t word = bp >> 5;
                uint32_t bit = 31u - (uint32_t)(bp & 31u);
                uint8_t* wp = out + off_st + 4ull * word;
                put32(wp, get32(wp) | (1u << bit));
              }
            }
          }
    }
  }
  if (p->lossless) {
    /* the fourth SZ stage over the finished stream, which ends the container */
    uint64_t raw = 4ull * swords;
    uint8_t* tmp = (uint8_t*)malloc(orc_lz_bound(raw));
    uint64_t lzb = orc_lz_encode(out + off_st, raw, tmp);
    uint64_t tot2 = al16(off_st + lzb);
    if (tot2 > cap) { free(tmp); ret = ORC_ERR_CAPACITY; goto done; }
    memset(out + off_st, 0, tot2 - off_st);
    memcpy(out + off_st, tmp, lzb);
    free(tmp);
    total = tot2;
    put64(out + 216, total);
    put32(out + 228, get32(out + 228) | ORC_FLAG_LOSSLESS);
    put64(out + 240, lzb);
    put32(out + 252, orc_crc32(out, 252));
  }
  *out_size = total;

  if (dump) {
    if (dump->dq) memcpy(dump->dq, dq, sizeof(int32_t) * n);
    if (dump->ok) memcpy(dump->ok, okv, n);
    if (dump->codes) memcpy(dump->codes, codes, sizeof(uint16_t) * g.nblocks * g.bvol);
    if (dump->nnflag) memcpy(dump->nnflag, nnf, g.nblocks);
    if (dump->hist) memcpy(dump->hist, hist, sizeof(uint64_t) * (size_t)nsym);
    if (dump->lens) memcpy(dump->lens, lens, (size_t)nsym);
  }
done:
  free(order); free(bbits); free(cw); free(lens); free(cz); free(dqb); free(okb); free(cn); free(vt); free(vc);
  free(hist); free(nout); free(nnf); free(codes); free(okv); free(dq);
  return ret;
}

/* ------------------------------------------------------------------------- */
/* Decompression (Section V): rebuild the canonical Huffman decoder, read the */
/* stream bit by bit, take balance points from their set, otherwise invert   */
/* the quantization and let the predictor walk the block from its start.     */
/* ------------------------------------------------------------------------- */
int orc_read_header(const uint8_t* in, uint64_t in_size, uint64_t dims[3], int* dtype) {
  if (in_size < O_HDR) return ORC_ERR_CORRUPT;
  if (memcmp(in, "PCMP", 4) != 0 || get32(in + 4) != 1) return ORC_ERR_CORRUPT;
  if (get32(in + 252) != orc_crc32(in, 252)) return ORC_ERR_CORRUPT;
  dims[0] = get64(in + 16); dims[1] = get64(in + 24); dims[2] = get64(in + 32);
  *dtype = (int)get32(in + 8);
  return ORC_OK;
}

int orc_decompress(const uint8_t* in, uint64_t in_size, void* xo, uint64_t cap_elems) {
  uint64_t dims[3];
  int dtype;
  int st = orc_read_header(in, in_size, dims, &dtype);
  if (st) return st;
  if (dtype != ORC_F32 && dtype != ORC_F64) return ORC_ERR_CORRUPT;
  size_t ts = dtype == ORC_F64 ? 8 : 4;
  int pred = (int)get32(in + 12);
  int block[3] = {(int)get32(in + 40), (int)get32(in + 44), (int)get32(in + 48)};
  int k = (int)get32(in + 52), h1 = (int)get32(in + 56), h2 = (int)get32(in + 60);
  int m = (int)get32(in + 64), s_in = (int)get32(in + 68);
  orc_consts c;
  memset(&c, 0, sizeof(c));
  c.dtype = dtype;
  c.Kp = (int32_t)get32(in + 100); c.Kn = (int32_t)get32(in + 104);
  c.Zq = (int32_t)get32(in + 108); c.S = (int32_t)get32(in + 112);
  uint32_t n_used = get32(in + 116);
  if (dtype == ORC_F32) {
    c.step32 = f_from_bits((uint32_t)get64(in + 120));
    c.inv32 = f_from_bits((uint32_t)get64(in + 128));
    c.ebdn32 = f_from_bits((uint32_t)get64(in + 136));
  } else {
    c.stepd = d_from_bits(get64(in + 120));
    c.invd = d_from_bits(get64(in + 128));
    c.ebdnd = d_from_bits(get64(in + 136));
  }
  uint64_t nblocks = get64(in + 144), n_out = get64(in + 152), swords = get64(in + 160);
  uint64_t off_w = get64(in + 168), off_cb = get64(in + 176), off_bb = get64(in + 184);
  uint64_t off_bn = get64(in + 192), off_ov = get64(in + 200), off_st = get64(in + 208);
  uint64_t total = get64(in + 216);
  int nw = (int)get32(in + 224);
  o_geom g;
  if (o_geom_make(dims, block, &g)) return ORC_ERR_CORRUPT;
  if (m < 2 || m > 16 || g.nblocks != nblocks || total > in_size) return ORC_ERR_CORRUPT;
  int wsz = pred == ORC_PRED_MLP_BF16 ? 8 : 4;
  if (pred == ORC_PRED_MLP || pred == ORC_PRED_MLP64 || pred == ORC_PRED_MLP_BF16) {
    if ((k != 7 && k != 13) || h1 < 1 || h1 > O_MAXH || h2 < 0 || h2 > O_MAXH || s_in < 0 || s_in > 30 ||
        nw != (pred != ORC_PRED_MLP_BF16 ? orc_mlp_nweights(k, h1, h2) : orc_qnet_len(k, h1, h2)))
      return ORC_ERR_CORRUPT;
  } else if (pred != ORC_PRED_LORENZO || nw != 0) {
    return ORC_ERR_CORRUPT;
  }
  uint32_t hflags = get32(in + 228);
  int lossless = (hflags & ORC_FLAG_LOSSLESS) != 0;
  uint64_t lzb = get64(in + 240);
  if (off_w + (uint64_t)wsz * nw > total || off_cb + 4ull * n_used > total || off_bb + 4ull * nblocks > total ||
      off_bn + 2ull * nblocks > total || off_ov + ts * n_out > total ||
      (lossless ? off_st + lzb > total : off_st + 4ull * swords > total))
    return ORC_ERR_CORRUPT;
  uint64_t n = dims[0] * dims[1] * dims[2];
  if (n > cap_elems) return ORC_ERR_CAPACITY;
  int nsym = 1 << m;
  int64_t R = (int64_t)1 << (m - 1);
  if (n_used > (uint32_t)nsym) return ORC_ERR_CORRUPT;

  float* wts = NULL;
  int64_t* qn = NULL;
  if (nw && (pred == ORC_PRED_MLP || pred == ORC_PRED_MLP64)) {
    wts = (float*)malloc(sizeof(float) * (size_t)nw);
    for (int i = 0; i < nw; i++) wts[i] = f_from_bits(get32(in + off_w + 4ull * i));
  }
  if (nw && pred == ORC_PRED_MLP_BF16) {
    /* the fixed-point network: shapes must match the header, shifts and
     * integers must lie in their stated ranges */
    qn = (int64_t*)malloc(sizeof(int64_t) * (size_t)nw);
    for (int i = 0; i < nw; i++) qn[i] = (int64_t)get64(in + off_w + 8ull * i);
    int bad = qn[0] != k || qn[1] != h1 || qn[2] != h2 || qn[3] != s_in;
    for (int i = 4; i < 7; i++) bad |= qn[i] < -30 || qn[i] > 30;
    for (int i = 7; i < 9; i++) bad |= qn[i] < 0 || qn[i] > 26;
    {
      int64_t F = qn[4] + qn[5] + qn[6] - qn[7] - qn[8];
      bad |= F < -20 || F > 62;
    }
    int li = O_QHDR;
    int lay[3][2] = {{h1, k}, {h2 ? h2 : 1, h1}, {h2 ? 1 : 0, h2}};
    for (int l = 0; l < 3 && !bad; l++) {
      for (int r = 0; r < lay[l][0]; r++) {
        for (int c2 = 0; c2 < lay[l][1]; c2++, li++) bad |= qn[li] < -255 || qn[li] > 255;
      }
      for (int r = 0; r < lay[l][0]; r++, li++) bad |= qn[li] < -1073741824LL || qn[li] > 1073741824LL;
    }
    if (bad || li != nw) { free(qn); return ORC_ERR_CORRUPT; }
  }
  /* canonical decoder tables: the stored list is the code order */
  uint8_t* lens = (uint8_t*)calloc((size_t)nsym, 1);
  int ret = ORC_OK;
  uint32_t cnt[O_LMAX + 1] = {0}, first[O_LMAX + 1] = {0}, offs[O_LMAX + 1] = {0};
  uint32_t* sorted = (uint32_t*)malloc(sizeof(uint32_t) * (n_used + 1));
  uint32_t prevl = 0;
  for (uint32_t t = 0; t < n_used; t++) {
    uint32_t e = get32(in + off_cb + 4ull * t);
    uint32_t s = e & 0xFFFFu, l = e >> 16;
    if (s >= (uint32_t)nsym || l < 1 || l > O_LMAX || lens[s] || l < prevl) { ret = ORC_ERR_CORRUPT; break; }
    lens[s] = (uint8_t)l;
    sorted[t] = s;
    cnt[l]++;
    prevl = l;
  }
  if (ret == ORC_OK) {
    uint32_t cc = 0, o = 0;
    for (int l = 1; l <= O_LMAX; l++) {
      cc = (cc + cnt[l - 1]) << 1;
      first[l] = cc;
      offs[l] = o;
      o += cnt[l];
      if (cnt[l] && (uint64_t)first[l] + cnt[l] > (1ull << l)) ret = ORC_ERR_CORRUPT;
    }
  }
  int32_t* dq = (int32_t*)malloc(sizeof(int32_t) * g.bvol);
  int32_t* vc = (int32_t*)malloc(sizeof(int32_t) * g.bvol);
  /* the paper-literal selection: real centred values, walked serially with drift */
  uint32_t flags = get32(in + 228);
  int lit = (flags & ORC_FLAG_LITERAL) != 0;
  if (lit && (dtype != ORC_F32 || pred == ORC_PRED_MLP_BF16 || pred == ORC_PRED_MLP64)) ret = ORC_ERR_CORRUPT;
  float* cvf = (float*)malloc(sizeof(float) * g.bvol);
  float ta = 0.0f;
  int64_t Ka = 0;
  /* the stream words: in place, or decoded from the lossless stage's section */
  const uint8_t* sbase = in + off_st;
  uint8_t* rawbuf = NULL;
  if (lossless && ret == ORC_OK) {
    rawbuf = (uint8_t*)malloc(4ull * swords + 16);
    if (orc_lz_decode(in + off_st, lzb, rawbuf, 4ull * swords)) ret = ORC_ERR_CORRUPT;
    sbase = rawbuf;
  }
  uint64_t bp = 0, oi = 0;
  uint64_t sbits = swords * 32ull;
  for (uint64_t b = 0; b < nblocks && ret == ORC_OK; b++) {
    uint32_t bw = get32(in + off_bb + 4ull * b);
    uint32_t nbits = bw & 0x7FFFFFFFu;
    int usen = (int)(bw >> 31);
    uint32_t no = (uint32_t)in[off_bn + 2ull * b] | ((uint32_t)in[off_bn + 2ull * b + 1] << 8);
    if (usen && !wts && !qn) { ret = ORC_ERR_CORRUPT; break; }
    uint64_t bend = bp + nbits;
    uint64_t oend = oi + no;
    if (bend > sbits || oend > n_out || no < 1) { ret = ORC_ERR_CORRUPT; break; }
    uint64_t bz = b / (g.nb[1] * g.nb[2]), by = (b / g.nb[2]) % g.nb[1], bx = b % g.nb[2];
    uint64_t o0 = bz * block[0], o1 = by * block[1], o2 = bx * block[2];
    int e0 = (int)((dims[0] - o0) < (uint64_t)block[0] ? dims[0] - o0 : (uint64_t)block[0]);
    int e1 = (int)((dims[1] - o1) < (uint64_t)block[1] ? dims[1] - o1 : (uint64_t)block[1]);
    int e2 = (int)((dims[2] - o2) < (uint64_t)block[2] ? dims[2] - o2 : (uint64_t)block[2]);
    int32_t da = 0;
    for (int lz = 0; lz < e0 && ret == ORC_OK; lz++)
      for (int ly = 0; ly < e1 && ret == ORC_OK; ly++)
        for (int lx = 0; lx < e2 && ret == ORC_OK; lx++) {
          int j = (lz * e1 + ly) * e2 + lx;
          uint64_t ig = ((o0 + lz) * dims[1] + (o1 + ly)) * dims[2] + (o2 + lx);
          uint32_t sym = 0;
          if (j > 0) {
            uint32_t code = 0;
            int found = 0;
            for (int l = 1; l <= O_LMAX; l++) {
              if (bp >= bend) break;
              uint32_t word = get32(sbase + 4ull * (bp >> 5));
              uint32_t bit = (word >> (31u - (uint32_t)(bp & 31u))) & 1u;
              bp++;
              code = (code << 1) | bit;
              if (cnt[l] && code - first[l] < cnt[l]) { sym = sorted[offs[l] + code - first[l]]; found = 1; break; }
            }
            if (!found) { ret = ORC_ERR_CORRUPT; break; }
          }
          if (lit) {
            float xv;
            if (j == 0 || sym == 0) {
              if (oi >= oend) { ret = ORC_ERR_CORRUPT; break; }
              memcpy(&xv, in + off_ov + ts * oi, 4);
              oi++;
              float t;
              int64_t K;
              o_realcode32(xv, &c, &t, &K);
              if (j == 0) { ta = t; Ka = K; }
              cvf[j] = o_clampf(o_cen(t, K, ta, Ka));
            } else {
              float pr = o_lit_pred(cvf, lz, ly, lx, e0, e1, e2, usen ? wts : NULL, k, h1, h2, s_in);
              float cc = pr + (float)((int64_t)sym - R);
              cvf[j] = o_clampf(cc);
              xv = o_lit_value(cc, ta, Ka, &c);
            }
            ((float*)xo)[ig] = xv;
            continue;
          }
          int32_t q;
          if (j == 0 || sym == 0) {
            if (oi >= oend) { ret = ORC_ERR_CORRUPT; break; }
            int ok;
            if (dtype == ORC_F32) {
              float v;
              memcpy(&v, in + off_ov + ts * oi, 4);
              ((float*)xo)[ig] = v;
              orc_transform32(v, &c, &q, &ok);
            } else {
              double v;
              memcpy(&v, in + off_ov + ts * oi, 8);
              ((double*)xo)[ig] = v;
              orc_transform64(v, &c, &q, &ok);
            }
            oi++;
            if (j == 0) da = q;
          } else {
            int32_t in7[7];
            for (int i = 0; i < 7; i++) {
              int qz = lz + O_S7[i][0], qy = ly + O_S7[i][1], qx = lx + O_S7[i][2];
              in7[i] = (qz >= 0 && qy >= 0 && qx >= 0) ? vc[(qz * e1 + qy) * e2 + qx] : 0;
            }
            int64_t pr;
            if (usen) {
              int32_t inn[13];
              for (int i = 0; i < k; i++) {
                int dz, dy, dx;
                o_stencil(k, i, &dz, &dy, &dx);
                int qz = lz + dz, qy = ly + dy, qx = lx + dx;
                inn[i] = (qz >= 0 && qy >= 0 && qx >= 0 && qz < e0 && qy < e1 && qx < e2)
                             ? vc[(qz * e1 + qy) * e2 + qx] : 0;
              }
              pr = qn ? orc_mlp_pred_q(qn, inn)
                      : (pred == ORC_PRED_MLP64 ? orc_mlp_pred64(wts, k, h1, h2, s_in, inn)
                                                : orc_mlp_pred32(wts, k, h1, h2, s_in, inn));
            } else {
              pr = o_lorenzo(in7);
            }
            int64_t qq = (int64_t)da + pr + ((int64_t)sym - R);
            if (qq > 2147483647LL || qq < -2147483647LL) { ret = ORC_ERR_CORRUPT; break; }
            q = (int32_t)qq;
            if (dtype == ORC_F32) ((float*)xo)[ig] = orc_recon32(q, &c);
            else ((double*)xo)[ig] = orc_recon64(q, &c);
          }
          dq[j] = q;
          int64_t v = (int64_t)q - (int64_t)da;
          vc[j] = (int32_t)(v > O_VCLAMP ? O_VCLAMP : (v < -O_VCLAMP ? -O_VCLAMP : v));
        }
    if (ret == ORC_OK && (bp != bend || oi != oend)) ret = ORC_ERR_CORRUPT;
  }
  free(rawbuf); free(cvf); free(vc); free(dq); free(sorted); free(lens); free(wts); free(qn);
  return ret;
}

/* ------------------------------------------------------------------------- */
/* Step a3: training (Section IV.C, Section V).                               */
/* Samples: a non-anchor point is drawn iff the high 32 bits of               */
/* mix64(seed, linear index) fall below thr32 (10% by default); it goes to    */
/* validation iff the low 32 bits mod 10 < 2 (the 8:2 split).  Samples are    */
/* listed in block order, then local raster order.  A sample is used for      */
/* learning only if the point, its anchor and its in-block stencil            */
/* neighbours share one non-zero sign class (Reading: the paper trains on    */
/* sampled blocks; sign and zero jumps are unpredictable balance points).     */
/* ------------------------------------------------------------------------- */
int orc_count_samples(const uint64_t dims[3], const int block[3], uint64_t seed, uint32_t thr32,
                      uint64_t* ntrain, uint64_t* nval) {
  o_geom g;
  if (o_geom_make(dims, block, &g)) return ORC_ERR_ARG;
  uint64_t nt = 0, nv = 0;
  for (uint64_t b = 0; b < g.nblocks; b++) {
    uint64_t bz = b / (g.nb[1] * g.nb[2]), by = (b / g.nb[2]) % g.nb[1], bx = b % g.nb[2];
    uint64_t o0 = bz * block[0], o1 = by * block[1], o2 = bx * block[2];
    for (uint64_t lz = 0; lz < (uint64_t)block[0] && o0 + lz < dims[0]; lz++)
      for (uint64_t ly = 0; ly < (uint64_t)block[1] && o1 + ly < dims[1]; ly++)
        for (uint64_t lx = 0; lx < (uint64_t)block[2] && o2 + lx < dims[2]; lx++) {
          if (lz == 0 && ly == 0 && lx == 0) continue;
          uint64_t ig = ((o0 + lz) * dims[1] + (o1 + ly)) * dims[2] + (o2 + lx);
          uint64_t h = orc_mix64(seed, ig);
          if ((uint32_t)(h >> 32) >= thr32) continue;
          if ((uint32_t)h % 10u < 2u) nv++; else nt++;
        }
  }
  *ntrain = nt;
  *nval = nv;
  return ORC_OK;
}

/* Gather: inputs [count][k] (clamped centred codes), target [count], use [count]. */
int orc_gather_samples(const void* x, const uint64_t dims[3], int dtype, const orc_consts* c,
                       const int block[3], int k, uint64_t seed, uint32_t thr32,
                       int32_t* tin, int32_t* ttg, uint8_t* tuse,
                       int32_t* vin, int32_t* vtg, uint8_t* vuse) {
  o_geom g;
  if (o_geom_make(dims, block, &g)) return ORC_ERR_ARG;
  uint64_t n = dims[0] * dims[1] * dims[2];
  int32_t* dq = (int32_t*)malloc(sizeof(int32_t) * n);
  for (uint64_t i = 0; i < n; i++) {
    int ok;
    if (dtype == ORC_F32) orc_transform32(((const float*)x)[i], c, &dq[i], &ok);
    else orc_transform64(((const double*)x)[i], c, &dq[i], &ok);
  }
  uint64_t it = 0, iv = 0;
  for (uint64_t b = 0; b < g.nblocks; b++) {
    uint64_t bz = b / (g.nb[1] * g.nb[2]), by = (b / g.nb[2]) % g.nb[1], bx = b % g.nb[2];
    uint64_t o0 = bz * block[0], o1 = by * block[1], o2 = bx * block[2];
    int e0 = (int)((dims[0] - o0) < (uint64_t)block[0] ? dims[0] - o0 : (uint64_t)block[0]);
    int e1 = (int)((dims[1] - o1) < (uint64_t)block[1] ? dims[1] - o1 : (uint64_t)block[1]);
    int e2 = (int)((dims[2] - o2) < (uint64_t)block[2] ? dims[2] - o2 : (uint64_t)block[2]);
    uint64_t ia = (o0 * dims[1] + o1) * dims[2] + o2;
    int32_t da = dq[ia];
    int ca = o_class(da, c);
    for (int lz = 0; lz < e0; lz++)
      for (int ly = 0; ly < e1; ly++)
        for (int lx = 0; lx < e2; lx++) {
          if (lz == 0 && ly == 0 && lx == 0) continue;
          uint64_t ig = ((o0 + lz) * dims[1] + (o1 + ly)) * dims[2] + (o2 + lx);
          uint64_t h = orc_mix64(seed, ig);
          if ((uint32_t)(h >> 32) >= thr32) continue;
          int isval = (uint32_t)h % 10u < 2u;
          int32_t* inp = isval ? vin + (size_t)iv * k : tin + (size_t)it * k;
          int cp = o_class(dq[ig], c);
          int use = cp != 0 && cp == ca;
          for (int i = 0; i < k; i++) {
            int dz, dy, dx;
            o_stencil(k, i, &dz, &dy, &dx);
            int qz = lz + dz, qy = ly + dy, qx = lx + dx;
            int32_t v = 0;
            if (qz >= 0 && qy >= 0 && qx >= 0 && qz < e0 && qy < e1 && qx < e2) {
              uint64_t iq = ((o0 + qz) * dims[1] + (o1 + qy)) * dims[2] + (o2 + qx);
              int64_t d = (int64_t)dq[iq] - (int64_t)da;
              v = (int32_t)(d > O_VCLAMP ? O_VCLAMP : (d < -O_VCLAMP ? -O_VCLAMP : d));
              if (o_class(dq[iq], c) != cp) use = 0;
            }
            inp[i] = v;
          }
          int64_t d = (int64_t)dq[ig] - (int64_t)da;
          int32_t tv = (int32_t)(d > O_VCLAMP ? O_VCLAMP : (d < -O_VCLAMP ? -O_VCLAMP : d));
          if (isval) { vtg[iv] = tv; vuse[iv] = (uint8_t)use; iv++; }
          else { ttg[it] = tv; tuse[it] = (uint8_t)use; it++; }
        }
  }
  free(dq);
  return ORC_OK;
}

/* Input scale: smallest s in [0, 30] with (sum min(t^2, 2^40)) >> 2s < n_used. */
int orc_input_shift(const int32_t* tg, const uint8_t* use, uint64_t n) {
  uint64_t s2 = 0, nu = 0;
  for (uint64_t i = 0; i < n; i++) {
    if (!use[i]) continue;
    uint64_t a = (uint64_t)((int64_t)tg[i] < 0 ? -(int64_t)tg[i] : (int64_t)tg[i]);
    uint64_t q = a * a;
    if (q > (1ull << 40)) q = 1ull << 40;
    s2 += q;
    nu++;
  }
  if (nu == 0) return 0;
  int s = 0;
  while (s < 30 && (s2 >> (2 * s)) >= nu) s++;
  return s;
}

/* Initial weights (Section IV.B): hidden units 0 and 1 take the +/- Lorenzo
 * weights with zero bias; with two hidden layers the pair is carried through
 * by [1,-1] and [-1,1]; the output takes (c, -c) with c = 1/(1+alpha)^L so that
 * the network equals Lorenzo.  Reading: the paper's "two numbers summing to
 * one" cannot give Lorenzo through a leaky ReLU; this pair does.  Other weights
 * of hidden layers start at small hash-derived values in [-2^-10, 2^-10); other
 * output weights and all other biases start at zero. */
void orc_init_weights(float* w, int k, int h1, int h2, uint64_t seed) {
  int nw = orc_mlp_nweights(k, h1, h2);
  for (int i = 0; i < nw; i++) w[i] = 0.0f;
  uint64_t ctr = 0;
  float* W1 = w;
  for (int j = 0; j < h1; j++)
    for (int i = 0; i < k; i++) {
      float val;
      if (j < 2 && h1 >= 2) val = (float)(j == 0 ? o_lz_weight(k, i) : -o_lz_weight(k, i));
      else val = (float)((int32_t)(orc_mix64(seed, ctr) >> 40) - 8388608) * 0x1p-33f;
      ctr++;
      W1[j * k + i] = val;
    }
  float* p = W1 + h1 * k + h1;
  float a1 = 1.0f + O_ALPHA;
  float cc;
  if (h2 > 0) {
    float* W2 = p;
    for (int j = 0; j < h2; j++)
      for (int i = 0; i < h1; i++) {
        float val;
        if (j < 2) val = (i == j) ? 1.0f : ((i < 2) ? -1.0f : 0.0f);
        else val = (float)((int32_t)(orc_mix64(seed, ctr) >> 40) - 8388608) * 0x1p-33f;
        ctr++;
        W2[j * h1 + i] = val;
      }
    p = W2 + h2 * h1 + h2;
    cc = 1.0f / (a1 * a1);
  } else {
    cc = 1.0f / a1;
  }
  p[0] = cc;
  p[1] = -cc;
}

#define O_BATCH 256

/* Pairwise tree sum over O_BATCH rows: level by level, element 2i + 2i+1. */
static float o_treesum(float* a) {
  for (int w = O_BATCH / 2; w >= 1; w /= 2)
    for (int i = 0; i < w; i++) a[i] = a[2 * i] + a[2 * i + 1];
  return a[0];
}

/* Gradient of the minibatch loss
 *   (1/B) sum_r use_r (o_r - t_r)^2   (+ L2 handled in the update)
 * with t_r = target_r 2^-s (targets in scaled units), B = rows.  Every
 * parameter's gradient is a pairwise tree sum of per-row terms (rows >= B
 * contribute +0). */
void orc_batch_grad(const float* w, int k, int h1, int h2, int s_in,
                    const int32_t* in, const int32_t* tg, const uint8_t* use, int B, float* g) {
  int nw = orc_mlp_nweights(k, h1, h2);
  int hl = h2 > 0 ? h2 : h1;
  float sig = ldexpf(1.0f, -s_in);
  const float* W1 = w;
  const float* b1 = W1 + h1 * k;
  const float* W2 = b1 + h1;
  const float* b2 = W2 + (h2 > 0 ? h2 * h1 : 0);
  const float* W3 = h2 > 0 ? b2 + h2 : W2;
  float ginv = 2.0f / (float)B;
  /* per-row terms for each parameter: [nw][O_BATCH] */
  float* terms = (float*)calloc((size_t)nw * O_BATCH, sizeof(float));
  for (int r = 0; r < B; r++) {
    float u[32], a1[O_MAXH], z1[O_MAXH], a2[O_MAXH], z2[O_MAXH], d2[O_MAXH], d1[O_MAXH];
    for (int i = 0; i < k; i++) u[i] = (float)in[(size_t)r * k + i] * sig;
    for (int j = 0; j < h1; j++) {
      float acc = b1[j];
      for (int i = 0; i < k; i++) acc = fmaf(W1[j * k + i], u[i], acc);
      z1[j] = acc;
      a1[j] = acc >= 0.0f ? acc : acc * O_ALPHA;
    }
    const float* hv = a1;
    if (h2 > 0) {
      for (int j = 0; j < h2; j++) {
        float acc = b2[j];
        for (int i = 0; i < h1; i++) acc = fmaf(W2[j * h1 + i], a1[i], acc);
        z2[j] = acc;
        a2[j] = acc >= 0.0f ? acc : acc * O_ALPHA;
      }
      hv = a2;
    }
    float o = W3[hl];
    for (int j = 0; j < hl; j++) o = fmaf(W3[j], hv[j], o);
    float t = (float)tg[r] * sig;
    float go = use[r] ? (o - t) * ginv : 0.0f;
    /* output layer */
    int base3 = (int)(W3 - w);
    for (int j = 0; j < hl; j++) terms[(size_t)(base3 + j) * O_BATCH + r] = go * hv[j];
    terms[(size_t)(base3 + hl) * O_BATCH + r] = go;
    float* dtop;
    if (h2 > 0) {
      for (int j = 0; j < h2; j++) {
        float tt = go * W3[j];
        d2[j] = z2[j] >= 0.0f ? tt : tt * O_ALPHA;
      }
      int baseW2 = (int)(W2 - w), baseb2 = (int)(b2 - w);
      for (int j = 0; j < h2; j++) {
        for (int i = 0; i < h1; i++) terms[(size_t)(baseW2 + j * h1 + i) * O_BATCH + r] = d2[j] * a1[i];
        terms[(size_t)(baseb2 + j) * O_BATCH + r] = d2[j];
      }
      for (int i = 0; i < h1; i++) {
        float s = 0.0f;
        for (int j = 0; j < h2; j++) s = fmaf(W2[j * h1 + i], d2[j], s);
        d1[i] = z1[i] >= 0.0f ? s : s * O_ALPHA;
      }
      dtop = d1;
    } else {
      for (int i = 0; i < h1; i++) {
        float tt = go * W3[i];
        d1[i] = z1[i] >= 0.0f ? tt : tt * O_ALPHA;
      }
      dtop = d1;
    }
    int baseb1 = (int)(b1 - w);
    for (int j = 0; j < h1; j++) {
      for (int i = 0; i < k; i++) terms[(size_t)(j * k + i) * O_BATCH + r] = dtop[j] * u[i];
      terms[(size_t)(baseb1 + j) * O_BATCH + r] = dtop[j];
    }
  }
  for (int q = 0; q < nw; q++) g[q] = o_treesum(terms + (size_t)q * O_BATCH);
  free(terms);
}

/* One SGD update: weights w <- w - lr (g + 2 lambda w); biases w <- w - lr g. */
void orc_sgd_update(float* w, const float* g, int k, int h1, int h2, float lr, float lam) {
  int nw = orc_mlp_nweights(k, h1, h2);
  int hl = h2 > 0 ? h2 : h1;
  float lam2 = lam + lam;
  for (int q = 0; q < nw; q++) {
    int isbias;
    if (q < h1 * k) isbias = 0;
    else if (q < h1 * k + h1) isbias = 1;
    else if (h2 > 0 && q < h1 * k + h1 + h2 * h1) isbias = 0;
    else if (h2 > 0 && q < h1 * k + h1 + h2 * h1 + h2) isbias = 1;
    else isbias = (q == nw - 1);
    (void)hl;
    if (isbias) {
      float u = lr * g[q];
      w[q] = w[q] - u;
    } else {
      float t = lam2 * w[q];
      float gt = g[q] + t;
      float u = lr * gt;
      w[q] = w[q] - u;
    }
  }
}

/* One epoch of minibatch SGD over the training list, in list order. */
void orc_train_epoch(float* w, int k, int h1, int h2, int s_in, const int32_t* in, const int32_t* tg,
                     const uint8_t* use, uint64_t n, float lr, float lam, uint64_t max_steps) {
  int nw = orc_mlp_nweights(k, h1, h2);
  float* g = (float*)malloc(sizeof(float) * (size_t)nw);
  uint64_t steps = 0;
  for (uint64_t s = 0; s < n && steps < max_steps; s += O_BATCH, steps++) {
    int B = (int)((n - s) < O_BATCH ? (n - s) : O_BATCH);
    orc_batch_grad(w, k, h1, h2, s_in, in + s * (uint64_t)k, tg + s, use + s, B, g);
    orc_sgd_update(w, g, k, h1, h2, lr, lam);
  }
  free(g);
}

/* Validation cost: sum of bitlen(min(|t - pred|, R)) over used samples;
 * w == NULL scores the Lorenzo predictor. */
uint64_t orc_val_cost(const float* w, int k, int h1, int h2, int s_in, const int32_t* in,
                      const int32_t* tg, const uint8_t* use, uint64_t n, int m) {
  int64_t R = (int64_t)1 << (m - 1);
  uint64_t cost = 0;
  for (uint64_t i = 0; i < n; i++) {
    if (!use[i]) continue;
    int64_t pr;
    if (w) {
      pr = orc_mlp_pred32(w, k, h1, h2, s_in, in + i * (uint64_t)k);
    } else {
      pr = 0;
      for (int j = 0; j < k; j++) pr += (int64_t)o_lz_weight(k, j) * in[i * (uint64_t)k + j];
    }
    int64_t d = (int64_t)tg[i] - pr;
    uint64_t a = (uint64_t)(d < 0 ? -d : d);
    cost += (uint64_t)o_bitlen(a < (uint64_t)R ? a : (uint64_t)R);
  }
  return cost;
}

/* Full training phase: gather, scale, train nmodels (lr, lambda) pairs from the
 * same initial weights, score on validation, choose.  Returns the chosen index
 * (-1 = Lorenzo). */
int orc_train(const void* x, const uint64_t dims[3], int dtype, double eb, const int block[3],
              int k, int h1, int h2, int m, uint64_t seed, uint32_t thr32, int nmodels,
              const float* lrs, const float* lams, float* w_out /* nmodels * nw */,
              int* s_in_out, uint64_t* costs /* nmodels + 1, last = Lorenzo */) {
  uint64_t n = dims[0] * dims[1] * dims[2];
  double amin, amax;
  int trivial;
  int st = orc_stats(x, n, dtype, &amin, &amax, &trivial);
  if (st) return st;
  orc_consts c;
  st = orc_make_consts(dtype, amin, amax, trivial, eb, &c);
  if (st) return st;
  uint64_t nt, nv;
  st = orc_count_samples(dims, block, seed, thr32, &nt, &nv);
  if (st) return st;
  int32_t* tin = (int32_t*)malloc(sizeof(int32_t) * (nt * k + 1));
  int32_t* ttg = (int32_t*)malloc(sizeof(int32_t) * (nt + 1));
  uint8_t* tus = (uint8_t*)malloc(nt + 1);
  int32_t* vin = (int32_t*)malloc(sizeof(int32_t) * (nv * k + 1));
  int32_t* vtg = (int32_t*)malloc(sizeof(int32_t) * (nv + 1));
  uint8_t* vus = (uint8_t*)malloc(nv + 1);
  orc_gather_samples(x, dims, dtype, &c, block, k, seed, thr32, tin, ttg, tus, vin, vtg, vus);
  int s_in = orc_input_shift(ttg, tus, nt);
  *s_in_out = s_in;
  int nw = orc_mlp_nweights(k, h1, h2);
  int best = -1;
  uint64_t lz = orc_val_cost(NULL, k, h1, h2, s_in, vin, vtg, vus, nv, m);
  costs[nmodels] = lz;
  uint64_t bestc = lz;
  for (int h = 0; h < nmodels; h++) {
    float* w = w_out + (size_t)h * nw;
    orc_init_weights(w, k, h1, h2, seed ^ 0x5DEECE66DULL);
    orc_train_epoch(w, k, h1, h2, s_in, tin, ttg, tus, nt, lrs[h], lams[h], ~0ull);
    costs[h] = orc_val_cost(w, k, h1, h2, s_in, vin, vtg, vus, nv, m);
    if (costs[h] < bestc) { bestc = costs[h]; best = h; }
  }
  free(tin); free(ttg); free(tus); free(vin); free(vtg); free(vus);
  return best;
}

/* Fixed-point form of a trained perceptron: gather the training phase's
 * samples again (same seed and rate) and build the qnet from weights w. */
int orc_quantize(const void* x, const uint64_t dims[3], int dtype, double eb, const int block[3],
                 int k, int h1, int h2, uint64_t seed, uint32_t thr32, const float* w, int s_in, int64_t* qnet) {
  uint64_t n = dims[0] * dims[1] * dims[2];
  double amin, amax;
  int trivial;
  int st = orc_stats(x, n, dtype, &amin, &amax, &trivial);
  if (st) return st;
  orc_consts c;
  st = orc_make_consts(dtype, amin, amax, trivial, eb, &c);
  if (st) return st;
  uint64_t nt, nv;
  st = orc_count_samples(dims, block, seed, thr32, &nt, &nv);
  if (st) return st;
  int32_t* tin = (int32_t*)malloc(sizeof(int32_t) * (nt * k + 1));
  int32_t* ttg = (int32_t*)malloc(sizeof(int32_t) * (nt + 1));
  uint8_t* tus = (uint8_t*)malloc(nt + 1);
  int32_t* vin = (int32_t*)malloc(sizeof(int32_t) * (nv * k + 1));
  int32_t* vtg = (int32_t*)malloc(sizeof(int32_t) * (nv + 1));
  uint8_t* vus = (uint8_t*)malloc(nv + 1);
  orc_gather_samples(x, dims, dtype, &c, block, k, seed, thr32, tin, ttg, tus, vin, vtg, vus);
  st = orc_qnet_build(w, k, h1, h2, s_in, tin, tus, nt, vin, vus, nv, qnet);
  free(tin); free(ttg); free(tus); free(vin); free(vtg); free(vus);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Report (not part of the method): prediction error of the FP32 and the      */
/* fixed-point perceptron against the same weights evaluated in FP64, and of  */
/* Lorenzo, over every non-anchor point of every block of a field, with the   */
/* inputs of the data-selection rule (Section IV.D, exact pre-quantized       */
/* codes).  out[0] = points; out[1..4] = sum of squared residuals (target     */
/* minus prediction) of Lorenzo, FP64, FP32, fixed point; out[5], out[6] =    */
/* sum of squared differences FP32 - FP64 and fixed point - FP64; out[7],     */
/* out[8] = points where FP32, fixed point differ from FP64; out[9..12] =     */
/* sum of bitlen(min(|residual|, R)) of the four predictors.  qnet may be     */
/* NULL (fixed-point entries stay 0).                                         */
/* ------------------------------------------------------------------------- */
int orc_pred_report(const void* x, const uint64_t dims[3], int dtype, double eb, const int block[3], int k, int h1,
                    int h2, int s_in, const float* w, const int64_t* qnet, int m, double out[13]) {
  for (int i = 0; i < 13; i++) out[i] = 0.0;
  if (dtype != ORC_F32 && dtype != ORC_F64) return ORC_ERR_DTYPE;
  if ((k != 7 && k != 13) || !w || m < 2 || m > 16) return ORC_ERR_ARG;
  o_geom g;
  if (o_geom_make(dims, block, &g)) return ORC_ERR_ARG;
  uint64_t n = dims[0] * dims[1] * dims[2];
  double amin, amax;
  int trivial;
  int st = orc_stats(x, n, dtype, &amin, &amax, &trivial);
  if (st) return st;
  orc_consts c;
  st = orc_make_consts(dtype, amin, amax, trivial, eb, &c);
  if (st) return st;
  int64_t R = (int64_t)1 << (m - 1);
  int32_t* dq = (int32_t*)malloc(sizeof(int32_t) * n);
  for (uint64_t i = 0; i < n; i++) {
    int ok;
    if (dtype == ORC_F32) orc_transform32(((const float*)x)[i], &c, &dq[i], &ok);
    else orc_transform64(((const double*)x)[i], &c, &dq[i], &ok);
  }
  int32_t* vc = (int32_t*)malloc(sizeof(int32_t) * g.bvol);
  int64_t* vt = (int64_t*)malloc(sizeof(int64_t) * g.bvol);
  for (uint64_t bz = 0; bz < g.nb[0]; bz++)
    for (uint64_t by = 0; by < g.nb[1]; by++)
      for (uint64_t bx = 0; bx < g.nb[2]; bx++) {
        uint64_t o0 = bz * block[0], o1 = by * block[1], o2 = bx * block[2];
        int e0 = (int)((dims[0] - o0) < (uint64_t)block[0] ? dims[0] - o0 : (uint64_t)block[0]);
        int e1 = (int)((dims[1] - o1) < (uint64_t)block[1] ? dims[1] - o1 : (uint64_t)block[1]);
        int e2 = (int)((dims[2] - o2) < (uint64_t)block[2] ? dims[2] - o2 : (uint64_t)block[2]);
        int32_t da = dq[(o0 * dims[1] + o1) * dims[2] + o2];
        for (int lz = 0; lz < e0; lz++)
          for (int ly = 0; ly < e1; ly++)
            for (int lx = 0; lx < e2; lx++) {
              int j = (lz * e1 + ly) * e2 + lx;
              int64_t v = (int64_t)dq[((o0 + lz) * dims[1] + (o1 + ly)) * dims[2] + (o2 + lx)] - (int64_t)da;
              vt[j] = v;
              vc[j] = (int32_t)(v > O_VCLAMP ? O_VCLAMP : (v < -O_VCLAMP ? -O_VCLAMP : v));
            }
        for (int lz = 0; lz < e0; lz++)
          for (int ly = 0; ly < e1; ly++)
            for (int lx = 0; lx < e2; lx++) {
              int j = (lz * e1 + ly) * e2 + lx;
              if (j == 0) continue;
              int32_t in7[7], in[13];
              for (int i = 0; i < 7; i++) {
                int qz = lz + O_S7[i][0], qy = ly + O_S7[i][1], qx = lx + O_S7[i][2];
                in7[i] = (qz >= 0 && qy >= 0 && qx >= 0) ? vc[(qz * e1 + qy) * e2 + qx] : 0;
              }
              for (int i = 0; i < k; i++) {
                int dz, dy, dx;
                o_stencil(k, i, &dz, &dy, &dx);
                int qz = lz + dz, qy = ly + dy, qx = lx + dx;
                in[i] = (qz >= 0 && qy >= 0 && qx >= 0 && qz < e0 && qy < e1 && qx < e2) ? vc[(qz * e1 + qy) * e2 + qx]
                                                                                          : 0;
              }
              int64_t pr[4];
              pr[0] = o_lorenzo(in7);
              pr[1] = orc_mlp_pred64(w, k, h1, h2, s_in, in);
              pr[2] = orc_mlp_pred32(w, k, h1, h2, s_in, in);
              pr[3] = qnet ? orc_mlp_pred_q(qnet, in) : pr[1];
              out[0] += 1.0;
              for (int f = 0; f < 4; f++) {
                double d = (double)(vt[j] - pr[f]);
                out[1 + f] += d * d;
                int64_t a = vt[j] - pr[f];
                a = a < 0 ? -a : a;
                out[9 + f] += (double)o_bitlen((uint64_t)(a < R ? a : R));
              }
              double d32 = (double)(pr[2] - pr[1]), dqv = (double)(pr[3] - pr[1]);
              out[5] += d32 * d32;
              out[6] += dqv * dqv;
              out[7] += pr[2] != pr[1];
              out[8] += pr[3] != pr[1];
            }
      }
  free(vt); free(vc); free(dq);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* The codes of block bi of a field exactly as orc_compress stores them, with */
/* the field's constants c (orc_stats + orc_make_consts of the whole field);  */
/* only the block's points are transformed.  A test aid that checks sampled   */
/* blocks of fields too large to compress here in full.  codes[j] for local   */
/* raster j < *npts (codes[0] = 0, the anchor); *usen = perceptron chosen.    */
/* ------------------------------------------------------------------------- */
int orc_block_codes(const void* x, const uint64_t dims[3], int dtype, const orc_consts* c, const orc_params* p,
                    uint64_t bi, uint16_t* codes, int* usen, int* npts) {
  if (dtype != ORC_F32 && dtype != ORC_F64) return ORC_ERR_DTYPE;
  if (p->m < 2 || p->m > 16) return ORC_ERR_ARG;
  o_geom g;
  if (o_geom_make(dims, p->block, &g)) return ORC_ERR_ARG;
  if (bi >= g.nblocks) return ORC_ERR_ARG;
  int use_q = p->pred == ORC_PRED_MLP_BF16 && p->qnet != NULL;
  int use_64 = p->pred == ORC_PRED_MLP64 && p->weights != NULL;
  int use_nn = ((p->pred == ORC_PRED_MLP || use_64) && p->weights != NULL) || use_q;
  int k = p->stencil;
  if (use_nn && (k != 7 && k != 13)) return ORC_ERR_ARG;
  int64_t R = (int64_t)1 << (p->m - 1);
  uint64_t bz = bi / (g.nb[1] * g.nb[2]), by = (bi / g.nb[2]) % g.nb[1], bx = bi % g.nb[2];
  uint64_t o0 = bz * p->block[0], o1 = by * p->block[1], o2 = bx * p->block[2];
  int e0 = (int)((dims[0] - o0) < (uint64_t)p->block[0] ? dims[0] - o0 : (uint64_t)p->block[0]);
  int e1 = (int)((dims[1] - o1) < (uint64_t)p->block[1] ? dims[1] - o1 : (uint64_t)p->block[1]);
  int e2 = (int)((dims[2] - o2) < (uint64_t)p->block[2] ? dims[2] - o2 : (uint64_t)p->block[2]);
  int np = e0 * e1 * e2;
  int32_t* dqb = (int32_t*)malloc(sizeof(int32_t) * (size_t)np);
  uint8_t* okb = (uint8_t*)malloc((size_t)np);
  int32_t* vc = (int32_t*)malloc(sizeof(int32_t) * (size_t)np);
  int64_t* vt = (int64_t*)malloc(sizeof(int64_t) * (size_t)np);
  uint16_t* cz = (uint16_t*)calloc((size_t)np, sizeof(uint16_t));
  uint16_t* cn = (uint16_t*)calloc((size_t)np, sizeof(uint16_t));
  for (int lz = 0; lz < e0; lz++)
    for (int ly = 0; ly < e1; ly++)
      for (int lx = 0; lx < e2; lx++) {
        int j = (lz * e1 + ly) * e2 + lx;
        uint64_t ig = ((o0 + lz) * dims[1] + (o1 + ly)) * dims[2] + (o2 + lx);
        int ok;
        if (dtype == ORC_F32) orc_transform32(((const float*)x)[ig], c, &dqb[j], &ok);
        else orc_transform64(((const double*)x)[ig], c, &dqb[j], &ok);
        okb[j] = (uint8_t)ok;
      }
  int un = o_block(dqb, okb, e0, e1, e2, p, use_nn, use_q, use_64, k, R, vc, vt, cz, cn);
  const uint16_t* cs = un ? cn : cz;
  codes[0] = 0;
  for (int j = 1; j < np; j++) codes[j] = cs[j];
  *usen = un;
  *npts = np;
  free(dqb); free(okb); free(vc); free(vt); free(cz); free(cn);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Section IV.C, model selection by simulated compression.  A predictor's     */
/* validation residuals are quantized as the compressor would (code k + R, or */
/* 0 for a balance point when |k| >= R), Huffman-coded with the code of their */
/* own histogram (orc_huffman_lengths, lmax 24), and every balance point adds */
/* its stored value (value_bits, 32 or 64).  Returns the simulated size in    */
/* bits; w == NULL scores Lorenzo.                                            */
/* ------------------------------------------------------------------------- */
/* The validation histogram of one predictor: every used sample's residual  */
/* quantized as the compressor would (code k + R, or 0 when |k| >= R).       */
void orc_val_hist(const float* w, int k, int h1, int h2, int s_in, const int32_t* in, const int32_t* tg,
                  const uint8_t* use, uint64_t n, int m, uint64_t* hist) {
  int nsym = 1 << m;
  int64_t R = (int64_t)1 << (m - 1);
  memset(hist, 0, sizeof(uint64_t) * (size_t)nsym);
  for (uint64_t i = 0; i < n; i++) {
    if (!use[i]) continue;
    int64_t pr;
    if (w) {
      pr = orc_mlp_pred32(w, k, h1, h2, s_in, in + i * (uint64_t)k);
    } else {
      pr = 0;
      for (int j = 0; j < k; j++) pr += (int64_t)o_lz_weight(k, j) * in[i * (uint64_t)k + j];
    }
    int64_t d = (int64_t)tg[i] - pr;
    int64_t a = d < 0 ? -d : d;
    hist[a <= R - 1 ? d + R : 0]++;
  }
}

uint64_t orc_val_size(const float* w, int k, int h1, int h2, int s_in, const int32_t* in, const int32_t* tg,
                      const uint8_t* use, uint64_t n, int m, int value_bits) {
  int nsym = 1 << m;
  uint64_t* hist = (uint64_t*)calloc((size_t)nsym, sizeof(uint64_t));
  uint8_t* lens = (uint8_t*)malloc((size_t)nsym);
  orc_val_hist(w, k, h1, h2, s_in, in, tg, use, n, m, hist);
  orc_huffman_lengths(hist, nsym, O_LMAX, lens, NULL);
  uint64_t bits = hist[0] * (uint64_t)value_bits;
  for (int c = 0; c < nsym; c++) bits += hist[c] * (uint64_t)lens[c];
  free(lens); free(hist);
  return bits;
}

/* ------------------------------------------------------------------------- */
/* Section IV.C, the Huffman code of the training phase: from the validation  */
/* set's code frequencies averaged per block, a Huffman tree whose code the   */
/* compression phase then uses directly.  Readings: averaging divides every   */
/* count by the same number of blocks, which leaves the Huffman construction  */
/* unchanged, so the totals are used; symbol 0 (the balance-point marker)     */
/* counts at least once, so that balance points stay codable whether or not  */
/* the sample held one.  The paper leaves codes the sample never saw without  */
/* a code word (they become balance points).  With span_fill, every code     */
/* between the smallest and the largest code the sample saw counts at least   */
/* once too, so that only codes beyond the sampled span become balance points */
/* (a variant of this build: a validation sample of a wide residual           */
/* distribution misses many codes inside its span).  Writes the list          */
/* (sym | len << 16, most frequent first) and returns its length.             */
/* ------------------------------------------------------------------------- */
int orc_sample_codebook(const uint64_t* hist, int m, int span_fill, uint32_t* list) {
  int nsym = 1 << m;
  uint64_t* h = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nsym);
  uint8_t* lens = (uint8_t*)malloc((size_t)nsym);
  uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nsym);
  memcpy(h, hist, sizeof(uint64_t) * (size_t)nsym);
  if (span_fill) {
    int lo = nsym, hi = 0;
    for (int c = 1; c < nsym; c++)
      if (h[c] > 0) { if (c < lo) lo = c; hi = c; }
    for (int c = lo; c <= hi; c++)
      if (h[c] == 0) h[c] = 1;
  }
  if (h[0] == 0) h[0] = 1;
  int n = orc_huffman_lengths(h, nsym, O_LMAX, lens, order);
  for (int t = 0; t < n; t++) list[t] = order[t] | ((uint32_t)lens[order[t]] << 16);
  free(order); free(lens); free(h);
  return n;
}

/* The sample codebook of a field for one predictor (FP32 weights w, or       */
/* Lorenzo when w is NULL): the validation samples are drawn as the training  */
/* phase draws them (seed, thr32), their residuals histogrammed at m code     */
/* bits, and the list built by orc_sample_codebook.  Returns its length, or a */
/* negative status.                                                           */
int orc_sample_codebook_for(const void* x, const uint64_t dims[3], int dtype, double eb, const int block[3], int k,
                            int h1, int h2, int s_in, const float* w, int m, uint64_t seed, uint32_t thr32,
                            int span_fill, uint32_t* list) {
  uint64_t n = dims[0] * dims[1] * dims[2];
  double amin, amax;
  int trivial;
  int st = orc_stats(x, n, dtype, &amin, &amax, &trivial);
  if (st) return st;
  orc_consts c;
  st = orc_make_consts(dtype, amin, amax, trivial, eb, &c);
  if (st) return st;
  uint64_t nt, nv;
  st = orc_count_samples(dims, block, seed, thr32, &nt, &nv);
  if (st) return st;
  int32_t* tin = (int32_t*)malloc(sizeof(int32_t) * (nt * k + 1));
  int32_t* ttg = (int32_t*)malloc(sizeof(int32_t) * (nt + 1));
  uint8_t* tus = (uint8_t*)malloc(nt + 1);
  int32_t* vin = (int32_t*)malloc(sizeof(int32_t) * (nv * k + 1));
  int32_t* vtg = (int32_t*)malloc(sizeof(int32_t) * (nv + 1));
  uint8_t* vus = (uint8_t*)malloc(nv + 1);
  uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) << m);
  orc_gather_samples(x, dims, dtype, &c, block, k, seed, thr32, tin, ttg, tus, vin, vtg, vus);
  orc_val_hist(w, k, h1, h2, s_in, vin, vtg, vus, nv, m, hist);
  int nl = orc_sample_codebook(hist, m, span_fill, list);
  free(hist); free(tin); free(ttg); free(tus); free(vin); free(vtg); free(vus);
  return nl;
}

/* Section IV.C, the coverage rule for m: coverage(m) is the fraction of the  */
/* used validation samples whose residual a code of m bits covers,            */
/* |k| <= 2^(m-1) - 1.  Reading: among m = 2..16 take the coverage closest to */
/* 50% when eb_rel < 1.5% and to 80% otherwise; a tie goes to the larger m.   */
int orc_coverage_m(const float* w, int k, int h1, int h2, int s_in, const int32_t* in, const int32_t* tg,
                   const uint8_t* use, uint64_t n, double eb) {
  uint64_t cnt[66] = {0};
  uint64_t used = 0;
  for (uint64_t i = 0; i < n; i++) {
    if (!use[i]) continue;
    int64_t pr;
    if (w) {
      pr = orc_mlp_pred32(w, k, h1, h2, s_in, in + i * (uint64_t)k);
    } else {
      pr = 0;
      for (int j = 0; j < k; j++) pr += (int64_t)o_lz_weight(k, j) * in[i * (uint64_t)k + j];
    }
    int64_t d = (int64_t)tg[i] - pr;
    cnt[o_bitlen((uint64_t)(d < 0 ? -d : d))]++;
    used++;
  }
  if (used == 0) return 16;
  double target = eb < 0.015 ? 0.5 : 0.8;
  int best = 16;
  double bestd = 2.0;
  for (int mm = 16; mm >= 2; mm--) {
    uint64_t cov = 0;
    for (int b = 0; b <= mm - 1; b++) cov += cnt[b];
    double dd = fabs((double)cov / (double)used - target);
    if (dd < bestd) { bestd = dd; best = mm; }
  }
  return best;
}

/* The training phase with the paper's selection (Section IV.C): train the   */
/* nmodels settings as orc_train does, keep the predictor (a model or        */
/* Lorenzo) with the smallest simulated size at the initial m (strictly      */
/* smaller; Lorenzo wins ties, then the lower index), then choose m by the    */
/* coverage rule for that predictor.  sizes[nmodels + 1] (last = Lorenzo).    */
int orc_train_select(const void* x, const uint64_t dims[3], int dtype, double eb, const int block[3], int k, int h1,
                     int h2, int m, uint64_t seed, uint32_t thr32, int nmodels, const float* lrs, const float* lams,
                     float* w_out, int* s_in_out, uint64_t* sizes, int* m_out) {
  uint64_t n = dims[0] * dims[1] * dims[2];
  double amin, amax;
  int trivial;
  int st = orc_stats(x, n, dtype, &amin, &amax, &trivial);
  if (st) return st;
  orc_consts c;
  st = orc_make_consts(dtype, amin, amax, trivial, eb, &c);
  if (st) return st;
  uint64_t nt, nv;
  st = orc_count_samples(dims, block, seed, thr32, &nt, &nv);
  if (st) return st;
  int32_t* tin = (int32_t*)malloc(sizeof(int32_t) * (nt * k + 1));
  int32_t* ttg = (int32_t*)malloc(sizeof(int32_t) * (nt + 1));
  uint8_t* tus = (uint8_t*)malloc(nt + 1);
  int32_t* vin = (int32_t*)malloc(sizeof(int32_t) * (nv * k + 1));
  int32_t* vtg = (int32_t*)malloc(sizeof(int32_t) * (nv + 1));
  uint8_t* vus = (uint8_t*)malloc(nv + 1);
  orc_gather_samples(x, dims, dtype, &c, block, k, seed, thr32, tin, ttg, tus, vin, vtg, vus);
  int s_in = orc_input_shift(ttg, tus, nt);
  *s_in_out = s_in;
  int nw = orc_mlp_nweights(k, h1, h2);
  int vbits = dtype == ORC_F64 ? 64 : 32;
  int best = -1;
  uint64_t lz = orc_val_size(NULL, k, h1, h2, s_in, vin, vtg, vus, nv, m, vbits);
  sizes[nmodels] = lz;
  uint64_t bestc = lz;
  for (int h = 0; h < nmodels; h++) {
    float* w = w_out + (size_t)h * nw;
    orc_init_weights(w, k, h1, h2, seed ^ 0x5DEECE66DULL);
    orc_train_epoch(w, k, h1, h2, s_in, tin, ttg, tus, nt, lrs[h], lams[h], ~0ull);
    sizes[h] = orc_val_size(w, k, h1, h2, s_in, vin, vtg, vus, nv, m, vbits);
    if (sizes[h] < bestc) { bestc = sizes[h]; best = h; }
  }
  *m_out = orc_coverage_m(best >= 0 ? w_out + (size_t)best * nw : NULL, k, h1, h2, s_in, vin, vtg, vus, nv, eb);
  free(tin); free(ttg); free(tus); free(vin); free(vtg); free(vus);
  return best;
}
