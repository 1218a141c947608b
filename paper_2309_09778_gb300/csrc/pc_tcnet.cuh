// The fixed-point perceptron (Section IV.B network, in the exact integer
// form of pc_qmlp.cuh) on the fifth-generation tensor cores: tiles of 128
// points, A operands written by the threads into shared memory, weights
// resident in shared memory, accumulators in TMEM.
//
// Exact evaluation with f16 limbs.  Every layer input x (a centred code
// clamped to +-65535, or a hidden activation in +-32767) is offset to
// x' = x + X0 >= 0 (X0 = 65536 or 32768) and split as x' = 512 hi + lo,
// 0 <= lo < 512, 0 <= hi < 256.  The A operands hold 1024 + hi and 1024 + lo
// as f16 (integers below 2048, exact; the bit pattern is 0x6400 | value).
// Weights |W| <= 255 are exact in f16, every product is exact in FP32 and every
// partial sum is an integer below 2^24 in magnitude (at most 32 terms of
// 255 * 1535), so the FP32 accumulation is exact in any order.  Per hidden
// unit u with weight sum s_u:
//   D_hi = 1024 s_u + sum W hi,  D_lo = 1024 s_u + sum W lo,
//   bits(D + (M - 1024 s_u)) = K0 + sum W limb   (M = 1.5 2^23, K0 = bits(M);
//                                                 |sum W limb| < 2^22)
//   A = sum W x + B = 512 hb + lb + (B - 513 K0 - X0 s_u)   (32-bit wrap-around)
// The requantization of pc_qmlp.cuh, clamp(rhu(leaky(A) 2^-t)), is
//   max((A + 2^(t-1)) >> t, (A + 2^(t+3)) >> (t + 4)) clamped to +-32767,
// which picks the first term for A >= 0 and the second for A < 0.  The
// output layer (one unit) runs on the CUDA cores in 32-bit integers.
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

#include "pc_qmlp.cuh"
#include "pc_tc.cuh"

namespace pc {

// Shared-memory network of hidden width H (both hidden layers), stencil K <= 16.
template <int H>
struct TcStage {
  uint16_t b1[H * 16];  // layer-1 weights, H x 16 (columns >= K are zero), core-matrix layout
  uint16_t b2[H * H];   // layer-2 weights, H x H
  float c1[H], c2[H];   // M - 1024 s_u
  int cp1[H], cn1[H], cp2[H], cn2[H];  // requantization offsets of the two branches
  int w3[H];
  int b3, t1, t2, F;
  int mul512;                  // 512, read at run time so that the limb merge stays one IMAD
  int pad0_;
  uint64_t mbar[2];            // one MMA-completion barrier per warpgroup
  unsigned int tmem;           // TMEM base column of this CTA
  int pad_[1];
};

constexpr unsigned int kTcK0 = 0x4B400000u;  // bits of 1.5 * 2^23

// byte offset of element (row, col) in a core-matrix tile of `rows` rows
__host__ __device__ constexpr int tc_off(int row, int col, int rows) {
  return (col >> 3) * (rows / 8) * 128 + (row >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2;
}

__device__ __forceinline__ uint16_t f16_of_small(long long w) {
  return __half_as_ushort(__float2half_rn((float)w));
}

// Requantization offsets: (B + half) - 513 K0 - X0 s, wrapped to 32 bits.
__device__ __forceinline__ int tc_offset(long long B, long long half, long long X0, long long s) {
  const unsigned long long v = (unsigned long long)(B + half - X0 * s) - 513ull * (unsigned long long)kTcK0;
  return (int)(unsigned int)(v & 0xFFFFFFFFull);
}

// Stage the network q (device memory, int64, layout of pc_qmlp.cuh) for
// stencil K and widths (H, H).  Called by every thread of the CTA.
template <int K, int H>
__device__ void tcnet_stage(const long long* __restrict__ q, TcStage<H>& S) {
  const long long* W1 = q + kQHdr;
  const long long* B1 = W1 + H * K;
  const long long* W2 = B1 + H;
  const long long* B2 = W2 + H * H;
  const long long* W3 = B2 + H;
  const long long* B3 = W3 + H;
  const int t1 = (int)q[7], t2 = (int)q[8];
  for (int i = threadIdx.x; i < H * 16; i += blockDim.x) {
    const int n = i / 16, c = i % 16;
    S.b1[tc_off(n, c, H) / 2] = f16_of_small(c < K ? W1[n * K + c] : 0);
  }
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
    const int n = i / H, c = i % H;
    S.b2[tc_off(n, c, H) / 2] = f16_of_small(W2[n * H + c]);
  }
  for (int u = threadIdx.x; u < H; u += blockDim.x) {
    long long s1 = 0, s2 = 0;
    for (int i = 0; i < K; ++i) s1 += W1[u * K + i];
    for (int i = 0; i < H; ++i) s2 += W2[u * H + i];
    S.c1[u] = (float)(12582912.0 - 1024.0 * (double)s1);  // exact: an even integer below 2^25
    S.c2[u] = (float)(12582912.0 - 1024.0 * (double)s2);
    const long long hp1 = (1ll << t1) >> 1, hn1 = (1ll << (t1 + 4)) >> 1;
    const long long hp2 = (1ll << t2) >> 1, hn2 = (1ll << (t2 + 4)) >> 1;
    S.cp1[u] = tc_offset(B1[u], hp1, 65536, s1);
    S.cn1[u] = tc_offset(B1[u], hn1, 65536, s1);
    S.cp2[u] = tc_offset(B2[u], hp2, 32768, s2);
    S.cn2[u] = tc_offset(B2[u], hn2, 32768, s2);
    S.w3[u] = (int)W3[u];
  }
  if (threadIdx.x == 0) {
    S.b3 = (int)B3[0];
    S.t1 = t1;
    S.t2 = t2;
    S.F = (int)(q[4] + q[5] + q[6] - q[7] - q[8]);
    S.mul512 = 512;
  }
}

// Two offset limbs of an input (|x| <= 65535) as f16 bit patterns: 0x6400 | value.
__device__ __forceinline__ void tc_in_limbs(int x, uint32_t& hi16, uint32_t& lo16) {
  const uint32_t v = (uint32_t)(x + 65536);
  hi16 = 0x6400u | (v >> 9);
  lo16 = 0x6400u | (v & 511u);
}

// Hidden-layer epilogue of 16 units (u0 .. u0 + 15) of this thread's point:
// from the two accumulator limbs to the clamped activations h[].
__device__ __forceinline__ void tc_requant16(const uint32_t (&dh)[16], const uint32_t (&dl)[16], const float* c,
                                             const int* cp, const int* cn, int t, int t4, int mul512, int (&h)[16]) {
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    // 32-bit wrap-around sums; the two branch arguments are the true values
    const uint32_t hb = __float_as_uint(__fadd_rn(__uint_as_float(dh[u]), c[u]));
    const uint32_t lb = __float_as_uint(__fadd_rn(__uint_as_float(dl[u]), c[u]));
    const uint32_t base = hb * (uint32_t)mul512 + lb;
    const int p = (int)(base + (uint32_t)cp[u]) >> t;
    const int n = (int)(base + (uint32_t)cn[u]) >> t4;
    h[u] = max(-kQAct, min(kQAct, max(p, n)));
  }
}

// Store 16 activations (units u0 .. u0 + 15, u0 a multiple of 16) of row r as
// the two limb tiles of the next layer: x' = x + 32768 = 512 hi + lo.
__device__ __forceinline__ void tc_store_act16(const int (&h)[16], uint8_t* a_hi, uint8_t* a_lo, int u0, int r) {
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // low 16 bits of both; x' = x ^ 0x8000 in 16 bits
      const uint32_t tw = __byte_perm((uint32_t)h[ch * 8 + 2 * i], (uint32_t)h[ch * 8 + 2 * i + 1], 0x5410);
      lw[i] = (tw & 0x01FF01FFu) | 0x64006400u;
      hw[i] = ((tw >> 9) & 0x007F007Fu) ^ 0x64406440u;
    }
    const int off = ((u0 >> 3) + ch) * 2048 + r * 16;
    *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Wait limit of one MMA completion (polls).
constexpr uint32_t kTcWait = 1u << 22;

// One tile of 128 points for the warpgroup `wg` (its 128 threads call this
// together; thread r = row r).  x[K]: this thread's stencil inputs (centred
// codes).  abuf: this warpgroup's A tiles, hi at abuf, lo at abuf + 128 H 2.
// tm: this warpgroup's TMEM columns (hi sums at tm, lo sums at tm + H).
// phase: this warpgroup's barrier parity, flipped at every completion.
// Returns the prediction clamp(rne(A_out 2^-F), +-2^30) in pred, and false if a
// wait on the tensor cores ran out.
template <int K, int H>
__device__ __forceinline__ bool tcnet_tile(TcStage<H>& S, uint8_t* abuf, uint32_t tm, int wg, int r,
                                           uint32_t& phase, const int (&x)[K], int mul512, int& pred) {
  static_assert(K <= 16 && (H == 16 || H == 32), "tile shape");
  uint8_t* a_hi = abuf;
  uint8_t* a_lo = abuf + 128 * H * 2;
  const uint32_t lane_off = (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16;
  constexpr uint32_t ID = tc::idesc_f16_f32(128, H);
  constexpr uint32_t LBO_B = (H / 8) * 128;
  bool ok = true;
  // layer 1 operands: 16 columns per limb (inputs K .. 15 carry zero weights)
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c0 = ch * 8 + 2 * i, c1 = c0 + 1;
      uint32_t h0 = 0x6400u, l0 = 0x6400u, h1 = 0x6400u, l1 = 0x6400u;
      if (c0 < K) tc_in_limbs(max(-kQIn, min(kQIn, x[c0])), h0, l0);
      if (c1 < K) tc_in_limbs(max(-kQIn, min(kQIn, x[c1])), h1, l1);
      hw[i] = h0 | (h1 << 16);
      lw[i] = l0 | (l1 << 16);
    }
    const int off = ch * 2048 + r * 16;
    *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  tc::bar_sync_wg(wg);
  if (r == 0) {
    tc::fence_after_sync();
    const uint64_t db = tc::desc_kmajor(tc::smem_u32(S.b1), LBO_B, 128);
    tc::mma_f16(tm, tc::desc_kmajor(tc::smem_u32(a_hi), 2048, 128), db, ID, false);
    tc::mma_f16(tm + H, tc::desc_kmajor(tc::smem_u32(a_lo), 2048, 128), db, ID, false);
    tc::mma_commit(&S.mbar[wg]);
  }
  ok &= tc::mbar_wait(&S.mbar[wg], phase, kTcWait);
  phase ^= 1u;
  tc::fence_after_sync();
  const int t1 = S.t1, t2 = S.t2;
#pragma unroll
  for (int hh = 0; hh < H / 16; ++hh) {
    uint32_t dh[16], dl[16];
    tmem_ld16(tm + lane_off + hh * 16, dh);
    tmem_ld16(tm + lane_off + H + hh * 16, dl);
    tc::tmem_ld_wait();
    int h[16];
    tc_requant16(dh, dl, S.c1 + hh * 16, S.cp1 + hh * 16, S.cn1 + hh * 16, t1, t1 + 4, mul512, h);
    tc_store_act16(h, a_hi, a_lo, hh * 16, r);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  tc::bar_sync_wg(wg);
  if (r == 0) {
    tc::fence_after_sync();
#pragma unroll
    for (int kk = 0; kk < H / 16; ++kk) {
      const uint64_t db = tc::desc_kmajor(tc::smem_u32(S.b2) + kk * 2 * LBO_B, LBO_B, 128);
      tc::mma_f16(tm, tc::desc_kmajor(tc::smem_u32(a_hi) + kk * 2 * 2048, 2048, 128), db, ID, kk > 0);
      tc::mma_f16(tm + H, tc::desc_kmajor(tc::smem_u32(a_lo) + kk * 2 * 2048, 2048, 128), db, ID, kk > 0);
    }
    tc::mma_commit(&S.mbar[wg]);
  }
  ok &= tc::mbar_wait(&S.mbar[wg], phase, kTcWait);
  phase ^= 1u;
  tc::fence_after_sync();
  int acc = 0;
#pragma unroll
  for (int hh = 0; hh < H / 16; ++hh) {
    uint32_t dh[16], dl[16];
    tmem_ld16(tm + lane_off + hh * 16, dh);
    tmem_ld16(tm + lane_off + H + hh * 16, dl);
    tc::tmem_ld_wait();
    int h[16];
    tc_requant16(dh, dl, S.c2 + hh * 16, S.cp2 + hh * 16, S.cn2 + hh * 16, t2, t2 + 4, mul512, h);
#pragma unroll
    for (int u = 0; u < 16; ++u) acc += S.w3[hh * 16 + u] * h[u];
  }
  // the TMEM columns are read: the next tile's MMAs may overwrite them once
  // its barrier has passed
  tc::fence_before_sync();
  long long o = rne_shift((long long)acc + S.b3, S.F);
  const long long lim = 1073741824ll;
  pred = (int)(o > lim ? lim : (o < -lim ? -lim : o));
  return ok;
}

}  // namespace pc

namespace pc {

// ---------------------------------------------------------------------------
// The same exact evaluation with warp-level MMAs (mma.sync m16n8k16, f16 in,
// f32 accumulate): a warp evaluates 16 points, each layer as two MMA sets
// (hi limbs, lo limbs) against one weight matrix.  With lane = 4 g + c the
// thread holds rows g and g + 8, columns 2c, 2c + 1 (+ 8) of A and of each
// 16 x 8 accumulator block; an accumulator block pair is the next layer's A
// fragment.  Used where waves are too narrow for 128-point tiles.
// ---------------------------------------------------------------------------
template <int H>
struct WStage {
  static constexpr int NB = H / 8;          // n-blocks of a layer
  static constexpr int F1 = NB * 64;        // layer-1 B fragments (one k-chunk of 16 inputs)
  static constexpr int F2 = (H / 16) * NB * 64;
  uint32_t frag[F1 + F2];
};

// B fragment words of one 16 x 8 block: b0 = (k 2c, 2c + 1; n g), b1 = (k 2c + 8, 2c + 9; n g)
template <int K, int H>
__device__ void wnet_stage(const long long* __restrict__ q, WStage<H>& W) {
  using S = WStage<H>;
  const long long* W1 = q + kQHdr;
  const long long* W2 = W1 + H * K + H;
  for (int f = threadIdx.x; f < S::F1 + S::F2; f += blockDim.x) {
    const bool l2 = f >= S::F1;
    const int r = l2 ? f - S::F1 : f;
    const int reg = r & 1, lane = (r >> 1) & 31, blk = r >> 6;
    const int g = lane >> 2, c = lane & 3;
    const int kc = l2 ? blk / S::NB : 0, nb = l2 ? blk % S::NB : blk;
    const int n = nb * 8 + g;
    const int k0 = kc * 16 + 2 * c + (reg ? 8 : 0);
    long long w0, w1;
    if (!l2) {
      w0 = k0 < K ? W1[n * K + k0] : 0;
      w1 = k0 + 1 < K ? W1[n * K + k0 + 1] : 0;
    } else {
      w0 = W2[n * H + k0];
      w1 = W2[n * H + k0 + 1];
    }
    W.frag[f] = (uint32_t)f16_of_small(w0) | ((uint32_t)f16_of_small(w1) << 16);
  }
}

__device__ __forceinline__ void mma_f16_sync(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One hidden-layer element: accumulator limbs to the clamped activation.
__device__ __forceinline__ int w_requant(float dh, float dl, float c, int cp, int cn, int t, int t4, int mul512) {
  const uint32_t hb = __float_as_uint(__fadd_rn(dh, c));
  const uint32_t lb = __float_as_uint(__fadd_rn(dl, c));
  const uint32_t base = hb * (uint32_t)mul512 + lb;
  const int p = (int)(base + (uint32_t)cp) >> t;
  const int n = (int)(base + (uint32_t)cn) >> t4;
  return max(-kQAct, min(kQAct, max(p, n)));
}

// Pack two activations (columns 2c, 2c + 1) as the next layer's hi and lo A words.
__device__ __forceinline__ void w_pack(int h0, int h1, uint32_t& hi, uint32_t& lo) {
  const uint32_t tw = __byte_perm((uint32_t)h0, (uint32_t)h1, 0x5410);
  lo = (tw & 0x01FF01FFu) | 0x64006400u;
  hi = ((tw >> 9) & 0x007F007Fu) ^ 0x64406440u;
}

// 16 points of a warp.  x[r][i]: this thread's inputs of row g (r = 0) and
// g + 8 (r = 1) at columns 2c, 2c + 1, 2c + 8, 2c + 9 (i = 0..3; columns >= K
// are ignored).  Returns the predictions of rows g and g + 8 in every lane of
// the quad.
template <int K, int H>
__device__ __forceinline__ void wnet_tile(const WStage<H>& W, const TcStage<H>& S, const int (&x)[2][4], int& pred0,
                                          int& pred1) {
  constexpr int NB = H / 8;
  const int lane = threadIdx.x & 31, c = lane & 3;
  const int mul512 = S.mul512;
  // layer 1: one k-chunk of 16 inputs
  uint32_t ah[4], al[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = q & 1, half = q >> 1;  // a[0]: row g cols 2c.., a[1]: row g+8, a[2]/a[3]: cols 2c+8..
    const int c0 = 2 * c + 8 * half;
    uint32_t h0 = 0x6400u, l0 = 0x6400u, h1 = 0x6400u, l1 = 0x6400u;
    if (c0 < K) tc_in_limbs(max(-kQIn, min(kQIn, x[r][2 * half])), h0, l0);
    if (c0 + 1 < K) tc_in_limbs(max(-kQIn, min(kQIn, x[r][2 * half + 1])), h1, l1);
    ah[q] = h0 | (h1 << 16);
    al[q] = l0 | (l1 << 16);
  }
  float dh[NB][4], dl[NB][4];
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    dh[nb][0] = dh[nb][1] = dh[nb][2] = dh[nb][3] = 0.0f;
    dl[nb][0] = dl[nb][1] = dl[nb][2] = dl[nb][3] = 0.0f;
    const uint2 b = reinterpret_cast<const uint2*>(W.frag)[nb * 32 + lane];
    mma_f16_sync(dh[nb], ah, b.x, b.y);
    mma_f16_sync(dl[nb], al, b.x, b.y);
  }
  int h[NB][4];
#pragma unroll
  for (int nb = 0; nb < NB; ++nb)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int u = nb * 8 + 2 * c + (e & 1);
      h[nb][e] = w_requant(dh[nb][e], dl[nb][e], S.c1[u], S.cp1[u], S.cn1[u], S.t1, S.t1 + 4, mul512);
    }
  // layer 2: k-chunk kc covers the units of n-blocks 2 kc and 2 kc + 1
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    dh[nb][0] = dh[nb][1] = dh[nb][2] = dh[nb][3] = 0.0f;
    dl[nb][0] = dl[nb][1] = dl[nb][2] = dl[nb][3] = 0.0f;
  }
#pragma unroll
  for (int kc = 0; kc < H / 16; ++kc) {
    w_pack(h[2 * kc][0], h[2 * kc][1], ah[0], al[0]);
    w_pack(h[2 * kc][2], h[2 * kc][3], ah[1], al[1]);
    w_pack(h[2 * kc + 1][0], h[2 * kc + 1][1], ah[2], al[2]);
    w_pack(h[2 * kc + 1][2], h[2 * kc + 1][3], ah[3], al[3]);
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      const uint2 b = reinterpret_cast<const uint2*>(W.frag + WStage<H>::F1)[(kc * NB + nb) * 32 + lane];
      mma_f16_sync(dh[nb], ah, b.x, b.y);
      mma_f16_sync(dl[nb], al, b.x, b.y);
    }
  }
  // layer 2 activations and the output unit on the CUDA cores: this thread's
  // units of rows g (e = 0, 1) and g + 8 (e = 2, 3), summed over the quad
  int acc0 = 0, acc1 = 0;
#pragma unroll
  for (int nb = 0; nb < NB; ++nb)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int u = nb * 8 + 2 * c + (e & 1);
      const int a = w_requant(dh[nb][e], dl[nb][e], S.c2[u], S.cp2[u], S.cn2[u], S.t2, S.t2 + 4, mul512);
      if (e < 2) acc0 += S.w3[u] * a;
      else acc1 += S.w3[u] * a;
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    acc0 += __shfl_xor_sync(0xFFFFFFFFu, acc0, o);
    acc1 += __shfl_xor_sync(0xFFFFFFFFu, acc1, o);
  }
  const long long lim = 1073741824ll;
  long long o0 = rne_shift((long long)acc0 + S.b3, S.F);
  long long o1 = rne_shift((long long)acc1 + S.b3, S.F);
  pred0 = (int)(o0 > lim ? lim : (o0 < -lim ? -lim : o0));
  pred1 = (int)(o1 > lim ? lim : (o1 < -lim ? -lim : o1));
}

}  // namespace pc
