// The paper-literal data selection (Section IV.D), an experimental mode for
// float32 fields: every point is predicted from the TRUE values of its causal
// in-block neighbours, which makes compression parallel point by point; the
// decoder can only predict from its own reconstructions, so errors accumulate
// (drift) until a balance point ("equilibrium point", a stored value) resets
// them.  The pointwise bound is not guaranteed in this mode.
//
// Real codes and arithmetic (every step an IEEE single operation, in this
// order):
//   - value x with the bound-safe transform's check passing and x != 0:
//     t = L(|x|) * inv (steps), K = the factor offset of its sign class;
//     otherwise t = 0, K = its integer code, and the point is always stored;
//   - centred on the block anchor: c = (t - t_a) + (K - K_a), clamped to
//     +-(2^24 - 1);
//   - prediction: Lorenzo sum of w_i c_i in stencil order, or the FP32
//     perceptron on u_i = c_i 2^-s with output o 2^s;
//   - residual k = rint(c - pred); code k + R when |k| <= R - 1, else 0; with
//     a period E > 0 the raster positions j = E, 2E, ... of each block are
//     stored as deliberate equilibrium points; every block uses the given
//     predictor;
//   - decoding: c' = pred(c'_nb) + k, z = c' + t_a, q' = rint(z) + K_a, value
//     0 in the zero class, else the class sign times exp2((z + K_a - K_cls) step).
// The decoder walks each block in wavefronts, which gives every point the
// same neighbour values as a serial raster walk.
#include "pc_kernels.cuh"
#include "pc_profile.cuh"

namespace pc {

constexpr int kLitHistWin = 2048;

struct LitCode {
  float t;
  long long K;
};

__device__ __forceinline__ LitCode lit_realcode(float x, const State& c, const Tabs& tb) {
  bool ok;
  const int q = Num<float>::transform(x, c, tb, ok);
  LitCode r;
  if (x != 0.0f && ok) {
    r.t = __fmul_rn(dev_log2f(fabsf(x), tb), c.inv32);
    r.K = x > 0.0f ? c.Kp : c.Kn;
  } else {
    r.t = 0.0f;
    r.K = q;
  }
  return r;
}

__device__ __forceinline__ bool lit_codable(float x, const State& c, const Tabs& tb) {
  bool ok;
  Num<float>::transform(x, c, tb, ok);
  return x != 0.0f && ok;
}

__device__ __forceinline__ float lit_clampf(float v) {
  return v > 16777215.0f ? 16777215.0f : (v < -16777215.0f ? -16777215.0f : v);
}

__device__ __forceinline__ float lit_cen(const LitCode& p, const LitCode& a) {
  return __fadd_rn(__fsub_rn(p.t, a.t), __ll2float_rn(p.K - a.K));
}

__device__ __forceinline__ long long lit_round(float r) {
  if (r != r) return 0;
  if (r > 1073741824.0f) r = 1073741824.0f;
  if (r < -1073741824.0f) r = -1073741824.0f;
  return (long long)rintf(r);
}

// FP32 perceptron on real centred inputs (the arithmetic of mlp_fwd with
// u_i = v_i 2^-s).
template <int K, int H1, int H2>
__device__ __forceinline__ float mlp_fwd_real(const Mlp& m, const float* v, float sig, float unsig) {
  float u[K];
#pragma unroll
  for (int i = 0; i < K; ++i) u[i] = __fmul_rn(v[i], sig);
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

// Prediction of (lz, ly, lx) from the centred values `get(qz, qy, qx)` of its
// causal in-block neighbours (0 outside the e0 x e1 x e2 block).  K == 0:
// Lorenzo.
template <int K, int H1, int H2, typename Get>
__device__ __forceinline__ float lit_pred(const Mlp& m, int lz, int ly, int lx, int e0, int e1, int e2, float sig,
                                          float unsig, Get get) {
  if constexpr (K == 0) {
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      const int qz = lz + s7_dz(i), qy = ly + s7_dy(i), qx = lx + s7_dx(i);
      const float v = (qz >= 0 && qy >= 0 && qx >= 0) ? get(qz, qy, qx) : 0.0f;
      acc = __fadd_rn(acc, __fmul_rn((float)lz_w(7, i), v));
    }
    return acc;
  } else {
    float in[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int qz = lz + st_dz(K, i), qy = ly + st_dy(K, i), qx = lx + st_dx(K, i);
      in[i] = (qz >= 0 && qy >= 0 && qx >= 0 && qz < e0 && qy < e1 && qx < e2) ? get(qz, qy, qx) : 0.0f;
    }
    return mlp_fwd_real<K, H1, H2>(m, in, sig, unsig);
  }
}

__device__ __forceinline__ float lit_value(float cc, const LitCode& a, const State& c, const Tabs& tb) {
  const float z = __fadd_rn(cc, a.t);
  long long q = lit_round(z) + a.K;
  if (q > 2147483647LL) q = 2147483647LL;
  if (q < -2147483647LL) q = -2147483647LL;
  const int cl = code_class((int)q, c);
  if (cl == 0) return 0.0f;
  const long long Kc = cl == 1 ? c.Kp : c.Kn;
  const float nr = __fadd_rn(z, __ll2float_rn(a.K - Kc));
  const float v = dev_exp2f(__fmul_rn(nr, c.step32), tb);
  return cl == 1 ? v : -v;
}

// Compression, one thread per point (block-strided padded raster order):
// codes, per-block balance counts and flags, histogram (shared window).
template <int K, int H1, int H2>
__global__ void __launch_bounds__(256) k_lit_compress(Geo g, const float* __restrict__ x, const State* __restrict__ st,
                                                      const Tabs* __restrict__ tabs, const __grid_constant__ Mlp mlp,
                                                      int eq_period, int m, uint16_t* codes, uint8_t* nnflag,
                                                      uint32_t* nout, unsigned long long* hist) {
  __shared__ Tabs tb;
  __shared__ unsigned int s_hist[kLitHistWin];
  for (int i = threadIdx.x; i < (int)(sizeof(Tabs) / 4); i += blockDim.x)
    reinterpret_cast<float*>(&tb)[i] = reinterpret_cast<const float*>(tabs)[i];
  __shared__ unsigned int s_hz;  // symbol 0: counted on chip, one atomic per CTA
  for (int i = threadIdx.x; i < kLitHistWin; i += blockDim.x) s_hist[i] = 0u;
  if (threadIdx.x == 0) s_hz = 0u;
  __syncthreads();
  const bool skip = st->err != 0;
  State c;
  c.Kp = st->Kp; c.Kn = st->Kn; c.Zq = st->Zq; c.S = st->S;
  c.step32 = st->step32; c.inv32 = st->inv32; c.ebdn32 = st->ebdn32;
  const int R = 1 << (m - 1);
  const int hbase = R - kLitHistWin / 2 > 0 ? R - kLitHistWin / 2 : 0;
  const float sig = K ? __uint_as_float((unsigned int)(127 - mlp.s_in) << 23) : 1.0f;
  const float unsig = K ? __uint_as_float((unsigned int)(127 + mlp.s_in) << 23) : 1.0f;
  const long long npad = g.nblocks * (long long)g.bvol;
  const int B1 = g.b[1], B2 = g.b[2];
  const long long n12 = g.n[1] * g.n[2];
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < npad && !skip;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / g.bvol;
    const int jp = (int)(idx - b * g.bvol);
    const long long bx = b % g.nb[2], byz = b / g.nb[2], by = byz % g.nb[1], bz = byz / g.nb[1];
    const long long z0 = bz * g.b[0], y0 = by * B1, x0 = bx * B2;
    const int e0 = (int)min((long long)g.b[0], g.n[0] - z0);
    const int e1 = (int)min((long long)B1, g.n[1] - y0);
    const int e2 = (int)min((long long)B2, g.n[2] - x0);
    const int lz = jp / (B1 * B2), ly = (jp / B2) % B1, lx = jp % B2;
    if (!(lz < e0 && ly < e1 && lx < e2)) {
      codes[idx] = 0;
      continue;
    }
    const float* org = x + z0 * n12 + y0 * g.n[2] + x0;
    if (jp == 0) {
      codes[idx] = 0;
      nnflag[b] = K ? 1 : 0;
      atomicAdd(&nout[b], 1u);
      continue;
    }
    const int jc = (lz * e1 + ly) * e2 + lx;
    const float xv = org[lz * n12 + ly * g.n[2] + lx];
    unsigned int code = 0;
    if (lit_codable(xv, c, tb) && !(eq_period > 0 && jc % eq_period == 0)) {
      const LitCode a = lit_realcode(org[0], c, tb);
      const float cp = lit_clampf(lit_cen(lit_realcode(xv, c, tb), a));
      auto get = [&](int qz, int qy, int qx) {
        return lit_clampf(lit_cen(lit_realcode(org[qz * n12 + qy * g.n[2] + qx], c, tb), a));
      };
      const float pr = lit_pred<K, H1, H2>(mlp, lz, ly, lx, e0, e1, e2, sig, unsig, get);
      const long long kk = lit_round(__fsub_rn(cp, pr));
      const long long ak = kk < 0 ? -kk : kk;
      code = ak <= R - 1 ? (unsigned int)(kk + R) : 0u;
    }
    codes[idx] = (uint16_t)code;
    const int hi = (int)code - hbase;
    if (code == 0) {
      atomicAdd(&nout[b], 1u);
      atomicAdd(&s_hz, 1u);
    } else if (hi >= 0 && hi < kLitHistWin) {
      atomicAdd(&s_hist[hi], 1u);
    } else {
      atomicAdd(&hist[code], 1ull);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kLitHistWin; i += blockDim.x)
    if (s_hist[i] && hbase + i < (1 << m)) atomicAdd(&hist[hbase + i], (unsigned long long)s_hist[i]);
  if (threadIdx.x == 0 && s_hz) atomicAdd(&hist[0], (unsigned long long)s_hz);
}

// Decoding, one warp per block: the block's wavefronts (z + y + x for the
// 7-point stencils, 4z + 2y + x for the 13-point one) one after another, the
// lanes over each wave's points; reconstructed centred values in shared memory.
constexpr int kLitWarps = 4;

template <int K, int H1, int H2>
__global__ void __launch_bounds__(32 * kLitWarps) k_lit_decode(Geo g, const uint8_t* __restrict__ in, DecInfo di,
                                                              DecScratch ds, float* __restrict__ xo,
                                                              const __grid_constant__ Mlp mlp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Tabs tb;
  const int BV = g.bvol, B1 = g.b[1], B2 = g.b[2];
  // wave lists (shared by the CTA), then per warp: centred values and balance ranks
  unsigned short* s_list = reinterpret_cast<unsigned short*>(smem);
  int* s_ws = reinterpret_cast<int*>(smem + ((2 * BV + 15) & ~15));
  const int nsched = 4 * (g.b[0] - 1) + 2 * (B1 - 1) + (B2 - 1) + 2;
  unsigned char* wbase = smem + ((2 * BV + 15) & ~15) + ((4 * (nsched + 1) + 15) & ~15);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* cv = reinterpret_cast<float*>(wbase + (size_t)wid * 6 * BV);
  unsigned short* rk = reinterpret_cast<unsigned short*>(cv + BV);
  for (int i = threadIdx.x; i < (int)(sizeof(Tabs) / 4); i += blockDim.x)
    reinterpret_cast<float*>(&tb)[i] = reinterpret_cast<const float*>(ds.ftab)[i];
  const bool s13 = K == 13;
  if (threadIdx.x == 0) {
    // counting sort of the raster positions by wave
    for (int sv = 0; sv <= nsched; ++sv) s_ws[sv] = 0;
    for (int j = 0; j < BV; ++j) {
      const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
      ++s_ws[(s13 ? 4 * lz + 2 * ly + lx : lz + ly + lx) + 1];
    }
    for (int sv = 1; sv <= nsched; ++sv) s_ws[sv] += s_ws[sv - 1];
    for (int j = 0; j < BV; ++j) {
      const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
      const int sv = s13 ? 4 * lz + 2 * ly + lx : lz + ly + lx;
      s_list[s_ws[sv + 1] - 1] = (unsigned short)j;  // filled from the end of each wave
      --s_ws[sv + 1];
    }
    // s_ws[sv + 1] now holds the start of wave sv; restore the ends
    for (int sv = 0; sv < nsched; ++sv) s_ws[sv] = s_ws[sv + 1];
    s_ws[nsched] = BV;
  }
  __syncthreads();
  if (*ds.err) return;
  State c;
  c.Kp = di.Kp; c.Kn = di.Kn; c.Zq = di.Zq; c.S = di.S;
  c.step32 = __uint_as_float((unsigned int)di.step_bits);
  c.inv32 = __uint_as_float((unsigned int)di.inv_bits);
  c.ebdn32 = __uint_as_float((unsigned int)di.ebdn_bits);
  const int R = 1 << (di.m - 1);
  const float sig = K ? __uint_as_float((unsigned int)(127 - mlp.s_in) << 23) : 1.0f;
  const float unsig = K ? __uint_as_float((unsigned int)(127 + mlp.s_in) << 23) : 1.0f;
  const float* ov = reinterpret_cast<const float*>(in + di.off_ov);
  const long long n12 = g.n[1] * g.n[2];
  const int nwave = s13 ? 4 * (g.b[0] - 1) + 2 * (B1 - 1) + (B2 - 1) + 1 : (g.b[0] - 1) + (B1 - 1) + (B2 - 1) + 1;
  bool bad = false;
  for (long long b = (long long)blockIdx.x * kLitWarps + wid; b < g.nblocks; b += (long long)gridDim.x * kLitWarps) {
    const long long bx = b % g.nb[2], byz = b / g.nb[2], by = byz % g.nb[1], bz = byz / g.nb[1];
    const long long z0 = bz * g.b[0], y0 = by * B1, x0 = bx * B2;
    const int e0 = (int)min((long long)g.b[0], g.n[0] - z0);
    const int e1 = (int)min((long long)B1, g.n[1] - y0);
    const int e2 = (int)min((long long)B2, g.n[2] - x0);
    const unsigned int no = *reinterpret_cast<const uint16_t*>(in + di.off_bn + 2ull * b);
    const bool usen = (*reinterpret_cast<const unsigned int*>(in + di.off_bb + 4ull * b)) >> 31;
    if (usen != (K != 0)) bad = true;
    const unsigned long long obase = ds.ooff[b];
    const uint16_t* cd = ds.codes + b * BV;
    // balance ranks in raster order (the anchor is rank 0)
    unsigned int run = 1;
    for (int j0 = 0; j0 < BV; j0 += 32) {
      const int j = j0 + lane;
      bool f = false;
      if (j < BV && j > 0) {
        const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
        f = lz < e0 && ly < e1 && lx < e2 && ds.sorted[cd[j]] == 0;
      }
      const unsigned int bal = __ballot_sync(0xFFFFFFFFu, f);
      if (f) rk[j] = (unsigned short)(run + __popc(bal & ((1u << lane) - 1u)));
      run += __popc(bal);
    }
    if (run != no || obase + no > di.n_out) bad = true;
    float* out = xo + z0 * n12 + y0 * g.n[2] + x0;
    const float xa = (obase < di.n_out) ? ov[obase] : 0.0f;
    const LitCode a = lit_realcode(xa, c, tb);
    if (lane == 0) {
      cv[0] = lit_clampf(lit_cen(a, a));
      out[0] = xa;
    }
    __syncwarp();
    for (int sw = 1; sw < nwave && !bad; ++sw) {
      for (int i = s_ws[sw] + lane; i < s_ws[sw + 1]; i += 32) {
        const int j = s_list[i];
        const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
        if (!(lz < e0 && ly < e1 && lx < e2)) continue;
        const unsigned int code = ds.sorted[cd[j]];
        float xv;
        if (code == 0) {
          const unsigned long long oi = obase + rk[j];
          xv = oi < di.n_out ? ov[oi] : 0.0f;
          cv[j] = lit_clampf(lit_cen(lit_realcode(xv, c, tb), a));
        } else {
          auto get = [&](int qz, int qy, int qx) { return cv[(qz * B1 + qy) * B2 + qx]; };
          const float pr = lit_pred<K, H1, H2>(mlp, lz, ly, lx, e0, e1, e2, sig, unsig, get);
          const float cc = __fadd_rn(pr, (float)((int)code - R));
          cv[j] = lit_clampf(cc);
          xv = lit_value(cc, a, c, tb);
        }
        out[lz * n12 + ly * g.n[2] + lx] = xv;
      }
      __syncwarp();
    }
  }
  if (bad) atomicExch(ds.err, PC_ERR_CORRUPT);
}

template <int K, int H1, int H2>
static int lit_compress_k(const float* x, const Geo& g, const State* st, const Tabs* tabs, const Mlp& mlp,
                          int eq_period, int m, uint16_t* codes, uint8_t* nnflag, uint32_t* nout,
                          unsigned long long* hist, int nsm, cudaStream_t s) {
  if (cudaMemsetAsync(nout, 0, 4ull * (size_t)g.nblocks, s) != cudaSuccess) return PC_ERR_CUDA;
  ProfScope p(kStCompress, s);
  k_lit_compress<K, H1, H2><<<(unsigned int)(nsm * 8), 256, 0, s>>>(g, x, st, tabs, mlp, eq_period, m, codes,
                                                                    nnflag, nout, hist);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

int launch_lit_compress(const float* x, const Geo& g, const State* st, const Tabs* tabs, const Mlp& mlp, int mode,
                        int eq_period, int m, uint16_t* codes, uint8_t* nnflag, uint32_t* nout,
                        unsigned long long* hist, int nsm, cudaStream_t s) {
  if (mode == 0) return lit_compress_k<0, 0, 0>(x, g, st, tabs, mlp, eq_period, m, codes, nnflag, nout, hist, nsm, s);
#define PC_LIT(KK, A, B)                                                                                            \
  if (mlp.k == KK && mlp.h1 == A && mlp.h2 == B)                                                                    \
    return lit_compress_k<KK, A, B>(x, g, st, tabs, mlp, eq_period, m, codes, nnflag, nout, hist, nsm, s);
  PC_LIT(7, 16, 16)
  PC_LIT(13, 32, 32)
  PC_LIT(7, 8, 8)
  PC_LIT(7, 2, 0)
  PC_LIT(13, 16, 16)
#undef PC_LIT
  return PC_ERR_ARG;
}

template <int K, int H1, int H2>
static int lit_decode_k(const uint8_t* in, const Geo& g, const DecInfo& di, const DecScratch& ds, const Mlp& mlp,
                        float* out, int nsm, cudaStream_t s) {
  const int nsched = 4 * (g.b[0] - 1) + 2 * (g.b[1] - 1) + (g.b[2] - 1) + 2;
  const size_t sm = ((2 * (size_t)g.bvol + 15) & ~(size_t)15) + ((4 * (size_t)(nsched + 1) + 15) & ~(size_t)15) +
                    (size_t)kLitWarps * 6 * g.bvol;
  auto kern = k_lit_decode<K, H1, H2>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return PC_ERR_CUDA;
  long long grid = (g.nblocks + kLitWarps - 1) / kLitWarps;
  if (grid > (long long)nsm * 16) grid = (long long)nsm * 16;
  ProfScope p(kStRecon, s);
  kern<<<(unsigned int)grid, 32 * kLitWarps, sm, s>>>(g, in, di, ds, out, mlp);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

int launch_lit_decode(const uint8_t* in, const Geo& g, const DecInfo& di, const DecScratch& ds, const Mlp& mlp,
                      float* out, int nsm, cudaStream_t s) {
  if (!di.usenn_any) return lit_decode_k<0, 0, 0>(in, g, di, ds, mlp, out, nsm, s);
#define PC_LIT(KK, A, B) \
  if (mlp.k == KK && mlp.h1 == A && mlp.h2 == B) return lit_decode_k<KK, A, B>(in, g, di, ds, mlp, out, nsm, s);
  PC_LIT(7, 16, 16)
  PC_LIT(13, 32, 32)
  PC_LIT(7, 8, 8)
  PC_LIT(7, 2, 0)
  PC_LIT(13, 16, 16)
#undef PC_LIT
  return PC_ERR_ARG;
}

}  // namespace pc
