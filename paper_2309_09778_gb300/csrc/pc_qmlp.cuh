// Fixed-point (BF16) perceptron on the tensor cores.
//
// The network (Section IV.B) in its fixed-point form: every weight of layer l
// is an integer |Wq| <= 255 times 2^-e_l (an exact bf16 value); the stencil
// inputs are the centred codes clamped to +-(2^16 - 1); hidden activations
// are integers clamped to +-(2^15 - 1):
//   A = sum Wq x + Bq;  hidden: Hq = clamp(rhu(leaky(A) 2^-t)), leaky(A) = A
//   for A >= 0 else A / 16, t >= 0;  output: pred = clamp(rne(A 2^-F), +-2^30)
// (rhu: round half up; rne: round half to even).  Sums stay below 2^28 and
// biases within 2^30, so the hidden layers run in 32-bit integers.
// On the tensor cores every input and activation is split into 8-bit limbs,
// x = 256 hi + lo with 0 <= lo < 256, and each layer is one bf16 GEMM against a
// block-diagonal weight matrix [[Wq^T, 0], [0, Wq^T]], so the hi and lo sums
// come out in separate columns.  Each product is bf16 x bf16, exact in FP32,
// and each column's sum is an integer of magnitude below 2^21, so the FP32
// accumulation is exact whatever the order inside the MMA; the two limb sums
// are combined in integer arithmetic: S = 256 S_hi + S_lo.
//
// MMA: mma.sync m16n8k16, bf16 inputs, f32 accumulate.  A warp evaluates a
// tile of 16 points (MMA rows).  With lane = 4 g + c: the thread holds rows g
// and g + 8, columns 2c, 2c + 1 (+8) of A and of each 16x8 accumulator block.
// The accumulator layout of one layer is the A-fragment layout of the next,
// so activations never leave the registers.
//
// qnet (int64, the container's weights section): k, h1, h2, s_in, e1, e2, e3,
// t1, t2, then W1[h1][k], B1[h1], W2[h2][h1], B2[h2], W3[h2], B3.
#pragma once
#include <cstdint>

#include "pc_device.cuh"

namespace pc {

constexpr int kQHdr = 9;
constexpr int kQIn = 65535;   // input clamp
constexpr int kQAct = 32767;  // activation clamp

__host__ __device__ constexpr int qnet_len(int k, int h1, int h2) {
  return kQHdr + h1 * k + h1 + (h2 ? h2 * h1 + h2 + h2 + 1 : h1 + 1);
}

// The network's stated ranges: shapes match, |W| <= 255, |B| <= 2^30,
// e in [-30, 30], t in [0, 26] (t + 4 <= 30 keeps the hidden shifts inside
// 32 bits), F = sum e - sum t in [-20, 62].  Checked on the host before
// compression and on the device before decompression.
__host__ __device__ inline bool qnet_valid(const long long* q, int k, int h1, int h2, int s_in) {
  if (q[0] != k || q[1] != h1 || q[2] != h2 || q[3] != s_in) return false;
  for (int i = 4; i < 7; ++i)
    if (q[i] < -30 || q[i] > 30) return false;
  for (int i = 7; i < 9; ++i)
    if (q[i] < 0 || q[i] > 26) return false;
  const long long F = q[4] + q[5] + q[6] - q[7] - q[8];
  if (F < -20 || F > 62) return false;
  int li = kQHdr;
  const int rows[3] = {h1, h2 ? h2 : 1, h2 ? 1 : 0};
  const int cols[3] = {k, h1, h2};
  for (int l = 0; l < 3; ++l) {
    for (int r = 0; r < rows[l] * cols[l]; ++r, ++li)
      if (q[li] < -255 || q[li] > 255) return false;
    for (int r = 0; r < rows[l]; ++r, ++li)
      if (q[li] < -(1ll << 30) || q[li] > (1ll << 30)) return false;
  }
  return li == qnet_len(k, h1, h2);
}

// Entry i of a network with the given shape is a weight (|W| <= 255) or a
// bias (|B| <= 2^30); the header entries (i < kQHdr) are checked by qnet_valid.
__host__ __device__ inline bool qnet_entry_ok(const long long* q, int i, int k, int h1, int h2) {
  const int rows[3] = {h1, h2 ? h2 : 1, h2 ? 1 : 0};
  const int cols[3] = {k, h1, h2};
  int base = kQHdr;
  for (int l = 0; l < 3; ++l) {
    const int nw = rows[l] * cols[l];
    if (i < base + nw) return q[i] >= -255 && q[i] <= 255;
    base += nw;
    if (i < base + rows[l]) return q[i] >= -(1ll << 30) && q[i] <= (1ll << 30);
    base += rows[l];
  }
  return true;
}

// rne(x 2^-s) for integer x: round to nearest, ties to even.
__device__ __forceinline__ long long rne_shift(long long x, int s) {
  if (s <= 0) return x * (1ll << (-s));
  if (s >= 62) return 0;
  const long long q = x >> s;  // floor (arithmetic shift)
  const long long r = x - (q << s);
  const long long h = 1ll << (s - 1);
  return q + ((r > h || (r == h && (q & 1))) ? 1 : 0);
}

// Hidden-layer requantization of an exact 32-bit sum (|a| < 2^30 + 2^28):
// rhu(leaky(a) 2^-t) = floor((a + h) 2^-s) with s = t (a >= 0) or t + 4,
// h = 2^(s-1) (0 for s = 0); clamp to +-(2^15 - 1).  hp/hn: the two halves.
__device__ __forceinline__ int leaky_requant32(int a, int t, int hp, int hn) {
  const bool neg = a < 0;
  const int h = (a + (neg ? hn : hp)) >> (neg ? t + 4 : t);
  return h > kQAct ? kQAct : (h < -kQAct ? -kQAct : h);
}

// 8-bit limbs: x = 256 hi + lo, 0 <= lo < 256 (hi in [-256, 255] for |x| <= 65535).
__device__ __forceinline__ void split_limbs(int x, int& hi, int& lo) {
  hi = x >> 8;
  lo = x & 255;
}

// Exact float of a small integer (|n| < 2^22) without a conversion
// instruction: adding 1.5 * 2^23 puts n in the low mantissa bits.
__device__ __forceinline__ float small_float(int n) { return __fsub_rn(__int_as_float(n + 0x4B400000), kMagic); }
// Integer of an exactly integral float (|v| < 2^22).
__device__ __forceinline__ int small_int(float v) { return __float_as_int(__fadd_rn(v, kMagic)) - 0x4B400000; }

// two small integers (|v| <= 256) as packed bf16 (exact: at most 8
// significant bits, so the float's low 16 bits are zero): low half = first
__device__ __forceinline__ uint32_t bf16x2_int(int a, int b) {
  return __byte_perm(__float_as_uint(small_float(a)), __float_as_uint(small_float(b)), 0x7632);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shapes of the three GEMMs for stencil K and widths H1, H2 (> 0).
template <int K, int H1, int H2>
struct QShape {
  static constexpr int KC1 = (2 * K + 15) / 16;  // k-chunks of layer 1 (limb columns, zero padded)
  static constexpr int NB1 = 2 * H1 / 8;         // n-blocks of layer 1 ([hi | lo] sums)
  static constexpr int KC2 = 2 * H1 / 16;
  static constexpr int NB2 = 2 * H2 / 8;
  static constexpr int KC3 = 2 * H2 / 16;
  // B fragments (two u32 per lane per (k-chunk, n-block))
  static constexpr int F1 = KC1 * NB1 * 64;
  static constexpr int F2 = KC2 * NB2 * 64;
  static constexpr int F3 = KC3 * 64;
  static constexpr int NFRAG = F1 + F2 + F3;
  static constexpr int NBIAS = H1 + H2 + 1;
};

// Scalars of the network.
struct QSc {
  int e1, e2, e3, t1, t2, F;
};

// Block-diagonal layer matrix entry B[c][n] (rows c: limb inputs, columns n:
// [hi sums | lo sums]) of a layer with nin inputs, nout outputs, weights Wq
// row-major [nout][nin]; returns the integer weight or 0.
__device__ __forceinline__ int qlayer_b(const long long* W, int nin, int nout, int c, int n) {
  if (c < nin && n < nout) return (int)W[n * nin + c];
  if (c >= nin && c < 2 * nin && n >= nout && n < 2 * nout) return (int)W[(n - nout) * nin + (c - nin)];
  return 0;
}
// Output layer: column 0 takes the hi limbs, column 1 the lo limbs.
__device__ __forceinline__ int qout_b(const long long* W, int nin, int c, int n) {
  if (n == 0 && c < nin) return (int)W[c];
  if (n == 1 && c >= nin && c < 2 * nin) return (int)W[c - nin];
  return 0;
}

// Stage the network from q (device memory) into shared memory: B fragments
// of the three GEMMs, the biases and the scalars.  Called by the whole CTA.
template <int K, int H1, int H2>
__device__ void qnet_stage(const long long* __restrict__ q, uint32_t* s_frag, long long* s_bias, QSc* s_sc) {
  using S = QShape<K, H1, H2>;
  const long long* W1 = q + kQHdr;
  const long long* B1 = W1 + H1 * K;
  const long long* W2 = B1 + H1;
  const long long* B2 = W2 + H2 * H1;
  const long long* W3 = B2 + H2;
  const long long* B3 = W3 + H2;
  // fragment word f: layer, (k-chunk, n-block), lane, which register
  for (int f = threadIdx.x; f < S::NFRAG; f += blockDim.x) {
    int r = f;
    int layer = 0;
    if (r >= S::F1) { r -= S::F1; layer = 1; }
    if (layer == 1 && r >= S::F2) { r -= S::F2; layer = 2; }
    const int reg = r & 1, lane = (r >> 1) & 31, blk = r >> 6;
    const int g = lane >> 2, c = lane & 3;
    const int nbs = layer == 0 ? S::NB1 : (layer == 1 ? S::NB2 : 1);
    const int kc = blk / nbs, nb = blk % nbs;
    const int n = nb * 8 + g;
    const int k0 = kc * 16 + 2 * c + (reg ? 8 : 0);
    int w0, w1;
    if (layer == 0) { w0 = qlayer_b(W1, K, H1, k0, n); w1 = qlayer_b(W1, K, H1, k0 + 1, n); }
    else if (layer == 1) { w0 = qlayer_b(W2, H1, H2, k0, n); w1 = qlayer_b(W2, H1, H2, k0 + 1, n); }
    else { w0 = qout_b(W3, H2, k0, n); w1 = qout_b(W3, H2, k0 + 1, n); }
    s_frag[f] = bf16x2_int(w0, w1);
  }
  for (int i = threadIdx.x; i < S::NBIAS; i += blockDim.x)
    s_bias[i] = i < H1 ? B1[i] : (i < H1 + H2 ? B2[i - H1] : B3[0]);
  if (threadIdx.x == 0) {
    QSc sc;
    sc.e1 = (int)q[4]; sc.e2 = (int)q[5]; sc.e3 = (int)q[6]; sc.t1 = (int)q[7]; sc.t2 = (int)q[8];
    sc.F = sc.e1 + sc.e2 + sc.e3 - sc.t1 - sc.t2;
    *s_sc = sc;
  }
}

// Layer-1 columns of this thread: for k-chunk kc and slot e (0..3), A-fragment
// column kc*16 + 2c + (e & 1) + 8 (e >> 1) is the hi limb of input i (col < K),
// the lo limb of input i = col - K (col < 2K), or zero padding.  qcol gives
// (input index, 1 for hi / 0 for lo), or input -1 for padding.
template <int K>
__device__ __forceinline__ void qcol(int kc, int e, int& input, int& hi) {
  const int c = threadIdx.x & 3;
  const int col = kc * 16 + 2 * c + (e & 1) + 8 * (e >> 1);
  input = col < K ? col : (col < 2 * K ? col - K : -1);
  hi = col < K ? 1 : 0;
}

// Limb value of slot (kc, e) from the clamped input x of that slot's input.
__device__ __forceinline__ int qlimb(int x, int hi) {
  int h, l;
  split_limbs(x, h, l);
  return hi ? h : l;
}

// One tile of 16 points.  lv[r][kc][e]: this thread's layer-1 limb values
// (qcol slot (kc, e)) for rows r = 0 (point g) and r = 1 (point g + 8).
// Returns the predictions of rows g and g + 8 in lanes with (lane & 3) == 0.
template <int K, int H1, int H2>
__device__ __forceinline__ void qnet_tile(const uint32_t* __restrict__ s_frag, const long long* __restrict__ s_bias,
                                          const QSc& sc, const int (&lv)[2][QShape<K, H1, H2>::KC1][4], int& pred0,
                                          int& pred1) {
  using S = QShape<K, H1, H2>;
  const int lane = threadIdx.x & 31, c = lane & 3;
  // layer 1: columns [hi(0..K-1) | lo(0..K-1) | 0]
  float d1[S::NB1][4];
#pragma unroll
  for (int nb = 0; nb < S::NB1; ++nb) d1[nb][0] = d1[nb][1] = d1[nb][2] = d1[nb][3] = 0.0f;
#pragma unroll
  for (int kc = 0; kc < S::KC1; ++kc) {
    uint32_t a[4];
    a[0] = bf16x2_int(lv[0][kc][0], lv[0][kc][1]);
    a[1] = bf16x2_int(lv[1][kc][0], lv[1][kc][1]);
    a[2] = bf16x2_int(lv[0][kc][2], lv[0][kc][3]);
    a[3] = bf16x2_int(lv[1][kc][2], lv[1][kc][3]);
#pragma unroll
    for (int nb = 0; nb < S::NB1; ++nb) {
      const uint2 b = reinterpret_cast<const uint2*>(s_frag)[(kc * S::NB1 + nb) * 32 + lane];
      mma_bf16(d1[nb], a, b.x, b.y);
    }
  }
  // combine limbs, bias, leaky ReLU, requantize: this thread's units are
  // n = 8 nb + 2 c + {0, 1} (nb < H1/8) for rows g (regs 0, 1) and g + 8 (2, 3)
  const int hp1 = (1 << sc.t1) >> 1, hn1 = (1 << (sc.t1 + 4)) >> 1;
  int h1v[S::NB1 / 2][4];
#pragma unroll
  for (int nb = 0; nb < S::NB1 / 2; ++nb)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int n = nb * 8 + 2 * c + (e & 1);
      const int sum = 256 * small_int(d1[nb][e]) + small_int(d1[nb + S::NB1 / 2][e]);
      h1v[nb][e] = leaky_requant32(sum + (int)s_bias[n], sc.t1, hp1, hn1);
    }
  // layer 2: A columns [hi(H1 units) | lo(H1 units)], straight from h1v
  float d2[S::NB2][4];
#pragma unroll
  for (int nb = 0; nb < S::NB2; ++nb) d2[nb][0] = d2[nb][1] = d2[nb][2] = d2[nb][3] = 0.0f;
#pragma unroll
  for (int kc = 0; kc < S::KC2; ++kc) {
    // k-chunk kc covers units 16 (kc mod (H1/16)) .. +15 of limb kc / (H1/16)
    const bool lo = kc >= H1 / 16;
    const int ub = (kc % (H1 / 16)) * 2;  // accumulator n-block holding those units
    uint32_t a[4];
    int hv[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int hh, ll;
      split_limbs(h1v[ub][e], hh, ll);
      hv[e] = lo ? ll : hh;
      split_limbs(h1v[ub + 1][e], hh, ll);
      hv[4 + e] = lo ? ll : hh;
    }
    a[0] = bf16x2_int(hv[0], hv[1]);
    a[1] = bf16x2_int(hv[2], hv[3]);
    a[2] = bf16x2_int(hv[4], hv[5]);
    a[3] = bf16x2_int(hv[6], hv[7]);
#pragma unroll
    for (int nb = 0; nb < S::NB2; ++nb) {
      const uint2 b = reinterpret_cast<const uint2*>(s_frag + S::F1)[(kc * S::NB2 + nb) * 32 + lane];
      mma_bf16(d2[nb], a, b.x, b.y);
    }
  }
  const int hp2 = (1 << sc.t2) >> 1, hn2 = (1 << (sc.t2 + 4)) >> 1;
  int h2v[S::NB2 / 2][4];
#pragma unroll
  for (int nb = 0; nb < S::NB2 / 2; ++nb)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int n = nb * 8 + 2 * c + (e & 1);
      const int sum = 256 * small_int(d2[nb][e]) + small_int(d2[nb + S::NB2 / 2][e]);
      h2v[nb][e] = leaky_requant32(sum + (int)s_bias[H1 + n], sc.t2, hp2, hn2);
    }
  // output: column 0 = hi sum, column 1 = lo sum
  float d3[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int kc = 0; kc < S::KC3; ++kc) {
    const bool lo = kc >= H2 / 16;
    const int ub = (kc % (H2 / 16)) * 2;
    uint32_t a[4];
    int hv[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int hh, ll;
      split_limbs(h2v[ub][e], hh, ll);
      hv[e] = lo ? ll : hh;
      split_limbs(h2v[ub + 1][e], hh, ll);
      hv[4 + e] = lo ? ll : hh;
    }
    a[0] = bf16x2_int(hv[0], hv[1]);
    a[1] = bf16x2_int(hv[2], hv[3]);
    a[2] = bf16x2_int(hv[4], hv[5]);
    a[3] = bf16x2_int(hv[6], hv[7]);
    const uint2 b = reinterpret_cast<const uint2*>(s_frag + S::F1 + S::F2)[kc * 32 + lane];
    mma_bf16(d3, a, b.x, b.y);
  }
  // lanes with c == 0 hold columns 0 (hi) and 1 (lo) of rows g and g + 8
  const long long bo = s_bias[H1 + H2];
  long long o0 = 256ll * small_int(d3[0]) + small_int(d3[1]) + bo;
  long long o1 = 256ll * small_int(d3[2]) + small_int(d3[3]) + bo;
  o0 = rne_shift(o0, sc.F);
  o1 = rne_shift(o1, sc.F);
  const long long lim = 1073741824ll;
  pred0 = (int)(o0 > lim ? lim : (o0 < -lim ? -lim : o0));
  pred1 = (int)(o1 > lim ? lim : (o1 < -lim ? -lim : o1));
}

}  // namespace pc
