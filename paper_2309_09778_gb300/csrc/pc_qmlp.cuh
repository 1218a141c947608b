// Fixed-point perceptron: the network's integer form shared by the training
// phase (quantization) and the tensor-core evaluators of pc_tcnet.cuh.
//
// The network (Section IV.B) in its fixed-point form: every weight of layer l
// is an integer |Wq| <= 255 times 2^-e_l (exact in f16 and bf16); the stencil
// inputs are the centred codes clamped to +-(2^16 - 1); hidden activations
// are integers clamped to +-(2^15 - 1):
//   A = sum Wq x + Bq;  hidden: Hq = clamp(rhu(leaky(A) 2^-t)), leaky(A) = A
//   for A >= 0 else A / 16, t >= 0;  output: pred = clamp(rne(A 2^-F), +-2^30)
// (rhu: round half up; rne: round half to even).  Sums stay below 2^28 and
// biases within 2^30, so the hidden layers run in 32-bit integers.
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

}  // namespace pc
