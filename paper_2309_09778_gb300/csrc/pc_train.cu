// a3: the training phase (Section IV.C) on the device.
//
//   k_samp_count   per block: how many points the hash draws for training /
//                  validation (non-anchor points, local raster order);
//   k_samp_scan    exclusive scans of those counts (one CTA);
//   k_samp_gather  per block: transform, stencil inputs, target and the
//                  "one sign class" use flag of every drawn point, written
//                  in block order;
//   k_in_shift     input scale s (sum of min(t^2, 2^40) over used samples);
//   k_init_w       Lorenzo-equal initial weights (Section IV.B);
//   k_train        a cluster of 8 CTAs per (lr, lambda) model: one epoch of
//                  minibatch SGD, every gradient a pairwise tree sum over the
//                  256 rows (32 rows per CTA, then the 8 CTA sums through
//                  distributed shared memory);
//   k_val          residual bit cost of every model and of Lorenzo on the
//                  validation samples;
//   k_choose       the cheapest model (Lorenzo unless strictly beaten).
#include <cooperative_groups.h>

#include "pc_kernels.cuh"
#include "pc_profile.cuh"
#include "pc_qmlp.cuh"

namespace pc {

__device__ __forceinline__ unsigned long long dev_mix64(unsigned long long seed, unsigned long long i) {
  // SplitMix64 output function on state seed + (i + 1) * golden gamma
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct TrainCtl {
  unsigned long long ntrain, nval, s2;
  unsigned long long nused;
  int s_in, chosen, err, pad;
};

// one warp per block
__global__ void __launch_bounds__(256) k_samp_count(Geo g, unsigned long long seed, unsigned int thr32,
                                                    unsigned int* cnt_t, unsigned int* cnt_v) {
  const long long b = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= g.nblocks) return;
  const long long bx = b % g.nb[2], t = b / g.nb[2], by = t % g.nb[1], bz = t / g.nb[1];
  const int e0 = (int)min((long long)g.b[0], g.n[0] - bz * g.b[0]);
  const int e1 = (int)min((long long)g.b[1], g.n[1] - by * g.b[1]);
  const int e2 = (int)min((long long)g.b[2], g.n[2] - bx * g.b[2]);
  unsigned int ct = 0, cv = 0;
  for (int j = lane; j < e0 * e1 * e2; j += 32) {
    if (j == 0) continue;
    const int lz = j / (e1 * e2), r = j % (e1 * e2), ly = r / e2, lx = r % e2;
    const unsigned long long lin =
        ((unsigned long long)(bz * g.b[0] + lz) * g.n[1] + (by * g.b[1] + ly)) * g.n[2] + bx * g.b[2] + lx;
    const unsigned long long h = dev_mix64(seed, lin);
    if ((unsigned int)(h >> 32) < thr32) {
      if ((unsigned int)h % 10u < 2u) ++cv; else ++ct;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ct += __shfl_xor_sync(0xFFFFFFFFu, ct, o);
    cv += __shfl_xor_sync(0xFFFFFFFFu, cv, o);
  }
  if (lane == 0) { cnt_t[b] = ct; cnt_v[b] = cv; }
}

// exclusive scans of both count arrays, one CTA (in place: counts -> offsets)
__global__ void __launch_bounds__(1024) k_samp_scan(long long nblocks, unsigned int* cnt_t, unsigned int* cnt_v,
                                                    unsigned long long* off_t, unsigned long long* off_v,
                                                    TrainCtl* ctl) {
  __shared__ unsigned long long s_w[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long per = (nblocks + nt - 1) / nt;
  const long long lo = min(nblocks, tid * per), hi = min(nblocks, lo + per);
  unsigned long long a = 0, bsum = 0;
  for (long long i = lo; i < hi; ++i) { a += cnt_t[i]; bsum += cnt_v[i]; }
  unsigned long long ta, tb;
  unsigned long long pa = cta_exscan<unsigned long long>(a, s_w, ta);
  unsigned long long pb = cta_exscan<unsigned long long>(bsum, s_w, tb);
  for (long long i = lo; i < hi; ++i) {
    off_t[i] = pa;
    off_v[i] = pb;
    pa += cnt_t[i];
    pb += cnt_v[i];
  }
  if (tid == 0) { ctl->ntrain = ta; ctl->nval = tb; }
}

// one warp per block; per-warp shared memory holds the block's codes
template <typename T>
__global__ void __launch_bounds__(128) k_samp_gather(const T* __restrict__ x, Geo g, const State* __restrict__ st,
                                                     const Tabs* __restrict__ tabs, unsigned long long seed,
                                                     unsigned int thr32, int k, const unsigned long long* off_t,
                                                     const unsigned long long* off_v, int* tin, int* ttg,
                                                     uint8_t* tus, int* vin, int* vtg, uint8_t* vus,
                                                     const TrainCtl* ctl, unsigned long long cap_t,
                                                     unsigned long long cap_v) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tabs& tb = *reinterpret_cast<Tabs*>(smem);
  int* s_dq = reinterpret_cast<int*>(smem + sizeof(Tabs)) + (threadIdx.x >> 5) * g.bvol;
  for (int i = threadIdx.x; i < (int)(sizeof(Tabs) / 4); i += blockDim.x)
    reinterpret_cast<float*>(&tb)[i] = reinterpret_cast<const float*>(tabs)[i];
  __syncthreads();
  if (st->err || ctl->ntrain > cap_t || ctl->nval > cap_v) return;
  State c;
  c.Kp = st->Kp; c.Kn = st->Kn; c.Zq = st->Zq; c.S = st->S;
  c.step32 = st->step32; c.inv32 = st->inv32; c.ebdn32 = st->ebdn32;
  c.stepd = st->stepd; c.invd = st->invd; c.ebdnd = st->ebdnd;
  const long long b = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= g.nblocks) return;
  const long long bx = b % g.nb[2], t = b / g.nb[2], by = t % g.nb[1], bz = t / g.nb[1];
  const int e0 = (int)min((long long)g.b[0], g.n[0] - bz * g.b[0]);
  const int e1 = (int)min((long long)g.b[1], g.n[1] - by * g.b[1]);
  const int e2 = (int)min((long long)g.b[2], g.n[2] - bx * g.b[2]);
  const int np = e0 * e1 * e2;
  const long long z0 = bz * g.b[0], y0 = by * g.b[1], x0 = bx * g.b[2];
  for (int j = lane; j < np; j += 32) {
    const int lz = j / (e1 * e2), r = j % (e1 * e2), ly = r / e2, lx = r % e2;
    bool okk;
    s_dq[j] = Num<T>::transform(x[((z0 + lz) * g.n[1] + (y0 + ly)) * g.n[2] + x0 + lx], c, tb, okk);
  }
  __syncwarp();
  const int da = s_dq[0];
  const int ca = code_class(da, c);
  unsigned long long ot = off_t[b], ovv = off_v[b];
  for (int j0 = 0; j0 < np; j0 += 32) {
    const int j = j0 + lane;
    bool selt = false, selv = false;
    unsigned long long h = 0;
    int lz = 0, ly = 0, lx = 0;
    if (j < np && j != 0) {
      lz = j / (e1 * e2);
      const int r = j % (e1 * e2);
      ly = r / e2;
      lx = r % e2;
      const unsigned long long lin = ((unsigned long long)(z0 + lz) * g.n[1] + (y0 + ly)) * g.n[2] + x0 + lx;
      h = dev_mix64(seed, lin);
      if ((unsigned int)(h >> 32) < thr32) {
        if ((unsigned int)h % 10u < 2u) selv = true; else selt = true;
      }
    }
    const unsigned int bt = __ballot_sync(0xFFFFFFFFu, selt), bv = __ballot_sync(0xFFFFFFFFu, selv);
    if (selt || selv) {
      const unsigned long long slot = selt ? ot + __popc(bt & ((1u << lane) - 1u)) : ovv + __popc(bv & ((1u << lane) - 1u));
      int* inp = selt ? tin + slot * (unsigned long long)k : vin + slot * (unsigned long long)k;
      const int cp = code_class(s_dq[j], c);
      bool use = cp != 0 && cp == ca;
      for (int i = 0; i < k; ++i) {
        const int qz = lz + st_dz(k, i), qy = ly + st_dy(k, i), qx = lx + st_dx(k, i);
        int v = 0;
        if (qz >= 0 && qy >= 0 && qx >= 0 && qz < e0 && qy < e1 && qx < e2) {
          const int q = s_dq[(qz * e1 + qy) * e2 + qx];
          v = clampd(q, da);
          if (code_class(q, c) != cp) use = false;
        }
        inp[i] = v;
      }
      const int tv = clampd(s_dq[j], da);
      if (selt) { ttg[slot] = tv; tus[slot] = use ? 1 : 0; }
      else { vtg[slot] = tv; vus[slot] = use ? 1 : 0; }
    }
    ot += __popc(bt);
    ovv += __popc(bv);
  }
}

__global__ void __launch_bounds__(256) k_in_shift(const int* __restrict__ ttg, const uint8_t* __restrict__ tus,
                                                  TrainCtl* ctl) {
  const unsigned long long n = ctl->ntrain;
  unsigned long long s2 = 0, nu = 0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    if (!tus[i]) continue;
    const long long t = ttg[i];
    const unsigned long long a = (unsigned long long)(t < 0 ? -t : t);
    unsigned long long q = a * a;
    if (q > (1ull << 40)) q = 1ull << 40;
    s2 += q;
    ++nu;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
    nu += __shfl_xor_sync(0xFFFFFFFFu, nu, o);
  }
  if ((threadIdx.x & 31) == 0 && (s2 || nu)) {
    atomicAdd(&ctl->s2, s2);
    atomicAdd(&ctl->nused, nu);
  }
}

// initial weights (Section IV.B): Lorenzo pair in hidden units 0 and 1, carried
// through the second hidden layer by [1,-1], [-1,1]; output (c, -c) with
// c = 1/(1+alpha)^L; other hidden-layer weights from the hash, others zero.
__global__ void k_init_w(float* w, int nmodels, int k, int h1, int h2, unsigned long long seed, TrainCtl* ctl) {
  const int nw = h1 * k + h1 + (h2 > 0 ? h2 * h1 + h2 : 0) + (h2 > 0 ? h2 : h1) + 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    const unsigned long long s2 = ctl->s2, nu = ctl->nused;
    int s = 0;
    if (nu) while (s < 30 && (s2 >> (2 * s)) >= nu) ++s;
    ctl->s_in = s;
  }
  if (p >= nw) return;
  auto noise = [&](unsigned long long ctr) {
    return __fmul_rn((float)((int)(dev_mix64(seed, ctr) >> 40) - 8388608), 0x1p-33f);
  };
  float v = 0.0f;
  const float a1 = __fadd_rn(1.0f, kAlpha);
  if (p < h1 * k) {
    const int j = p / k, i = p % k;
    if (j < 2 && h1 >= 2) v = (float)(j == 0 ? lz_w(k, i) : -lz_w(k, i));
    else v = noise((unsigned long long)p);
  } else if (h2 > 0 && p >= h1 * k + h1 && p < h1 * k + h1 + h2 * h1) {
    const int q = p - (h1 * k + h1), j = q / h1, i = q % h1;
    if (j < 2) v = (i == j) ? 1.0f : ((i < 2) ? -1.0f : 0.0f);
    else v = noise((unsigned long long)(h1 * k + q));
  } else {
    const int p3 = h1 * k + h1 + (h2 > 0 ? h2 * h1 + h2 : 0);
    const float cc = h2 > 0 ? __fdiv_rn(1.0f, __fmul_rn(a1, a1)) : __fdiv_rn(1.0f, a1);
    if (p == p3) v = cc;
    else if (p == p3 + 1) v = -cc;
  }
  for (int m = 0; m < nmodels; ++m) w[(size_t)m * nw + p] = v;
}

// One epoch of minibatch SGD per (lr, lambda) model (Section IV.C), each model
// on a cluster of 8 CTAs: CTA c of the cluster takes rows 32c .. 32c + 31 of
// every 256-row minibatch.  Its warps run the forward and backward passes of
// those rows (lane = row, the hidden units split over the warps) and leave
// every row's inputs, activations and deltas in shared memory; the CTA then
// sums each parameter's 32 row terms over a pairwise tree in row
// order ((r0 + r1) + (r2 + r3)) + ...; after a cluster barrier CTA c adds the
// eight CTA sums of its slice of the parameters pairwise, ((q0 + q1) +
// (q2 + q3)) + ((q4 + q5) + (q6 + q7)), updates them and writes the new
// values into every CTA's copy of the weights (distributed shared memory);
// a second cluster barrier ends the step.  The gradient is therefore the
// same balanced pairwise tree over the minibatch's 256 rows, in row order.
constexpr int kTrainCluster = 8;
constexpr int kTrainRows = 32;   // rows per CTA
constexpr int kTrainWarps = 8;   // warps per CTA: hidden units of the row phase, parameters of the sums

template <int K, int H1, int H2>
__global__ void __cluster_dims__(kTrainCluster, 1, 1) __launch_bounds__(32 * kTrainWarps)
    k_train(const int* __restrict__ tin, const int* __restrict__ ttg, const uint8_t* __restrict__ tus,
            float* __restrict__ wbuf, const float* __restrict__ lrs, const float* __restrict__ lams,
            const TrainCtl* __restrict__ ctl) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  constexpr int HL = H2 > 0 ? H2 : H1;
  constexpr int H2E = H2 > 0 ? H2 : 1;
  constexpr int NW = H1 * K + H1 + (H2 > 0 ? H2 * H1 + H2 : 0) + HL + 1;
  constexpr int OB1 = H1 * K, OW2 = OB1 + H1, OB2 = OW2 + H2 * H1, OW3 = H2 > 0 ? OB2 + H2 : OW2;
  // per-row vector: u[K] | a1[H1] | a2[H2] | d1[H1] | d2[H2] | go | 1
  constexpr int VA1 = K, VA2 = VA1 + H1, VD1 = VA2 + H2, VD2 = VD1 + H1, VGO = VD2 + H2, VONE = VGO + 1;
  constexpr int VS = (VONE + 1) | 1;  // odd row stride
  constexpr int SL = (NW + kTrainCluster - 1) / kTrainCluster;
  __shared__ float w[NW];
  __shared__ float part[NW];
  __shared__ float V[kTrainRows * VS];
  __shared__ unsigned short fa[NW], fb[NW];
  const int rank = (int)cl.block_rank();
  const int model = blockIdx.x / kTrainCluster;
  const int tid = threadIdx.x;
  float* wm = wbuf + (size_t)model * NW;
  for (int p = tid; p < NW; p += blockDim.x) {
    w[p] = wm[p];
    // the two row-vector entries whose product is parameter p's row term
    int a, b;
    if (p < OB1) { a = VD1 + p / K; b = p % K; }
    else if (p < OW2) { a = VD1 + (p - OB1); b = VONE; }
    else if (H2 > 0 && p < OB2) { a = VD2 + (p - OW2) / H1; b = VA1 + (p - OW2) % H1; }
    else if (H2 > 0 && p < OW3) { a = VD2 + (p - OB2); b = VONE; }
    else if (p < OW3 + HL) { a = VGO; b = (H2 > 0 ? VA2 : VA1) + (p - OW3); }
    else { a = VGO; b = VONE; }
    fa[p] = (unsigned short)a;
    fb[p] = (unsigned short)b;
  }
  const float lr = lrs[model], lam2 = __fadd_rn(lams[model], lams[model]);
  const int s_in = ctl->s_in;
  const float sig = __uint_as_float((unsigned int)(127 - s_in) << 23);
  const unsigned long long n = ctl->ntrain;
  float* const peer_part[kTrainCluster] = {
      cl.map_shared_rank(part, 0), cl.map_shared_rank(part, 1), cl.map_shared_rank(part, 2),
      cl.map_shared_rank(part, 3), cl.map_shared_rank(part, 4), cl.map_shared_rank(part, 5),
      cl.map_shared_rank(part, 6), cl.map_shared_rank(part, 7)};
  float* const peer_w[kTrainCluster] = {
      cl.map_shared_rank(w, 0), cl.map_shared_rank(w, 1), cl.map_shared_rank(w, 2), cl.map_shared_rank(w, 3),
      cl.map_shared_rank(w, 4), cl.map_shared_rank(w, 5), cl.map_shared_rank(w, 6), cl.map_shared_rank(w, 7)};
  __syncthreads();
  for (unsigned long long s0 = 0; s0 < n; s0 += 256) {
    const int B = (int)((n - s0) < 256ull ? (n - s0) : 256ull);
    // forward and backward of the CTA's 32 rows (lane = row), the hidden units
    // split over the warps; each unit's sums run in the same order as a single
    // thread's would
    {
      const int lane = tid & 31, q = tid >> 5;
      const int lrow = rank * kTrainRows + lane;
      const bool valid = lrow < B;
      const unsigned long long r = s0 + (valid ? lrow : 0);
      float* v = V + lane * VS;
      constexpr int NU1 = (H1 + kTrainWarps - 1) / kTrainWarps, NU2 = (H2E + kTrainWarps - 1) / kTrainWarps;
      float u[K], z1[NU1], z2[NU2];
#pragma unroll
      for (int i = 0; i < K; ++i) u[i] = valid ? __fmul_rn(small_int_to_float(tin[r * K + i]), sig) : 0.0f;
#pragma unroll
      for (int jj = 0; jj < NU1; ++jj) {
        const int j = q * NU1 + jj;
        if (j < H1) {
          float acc = w[OB1 + j];
#pragma unroll
          for (int i = 0; i < K; ++i) acc = __fmaf_rn(w[j * K + i], u[i], acc);
          z1[jj] = acc;
          v[VA1 + j] = valid ? (acc >= 0.0f ? acc : __fmul_rn(acc, kAlpha)) : 0.0f;
        }
      }
      if (q == 0) {
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = u[i];
      }
      __syncthreads();
      if constexpr (H2 > 0) {
#pragma unroll
        for (int jj = 0; jj < NU2; ++jj) {
          const int j = q * NU2 + jj;
          if (j < H2) {
            float acc = w[OB2 + j];
#pragma unroll 8
            for (int i = 0; i < H1; ++i) acc = __fmaf_rn(w[OW2 + j * H1 + i], v[VA1 + i], acc);
            z2[jj] = acc;
            v[VA2 + j] = valid ? (acc >= 0.0f ? acc : __fmul_rn(acc, kAlpha)) : 0.0f;
          }
        }
        __syncthreads();
      }
      if (q == 0) {
        float o = w[OW3 + HL];
#pragma unroll 8
        for (int j = 0; j < HL; ++j) o = __fmaf_rn(w[OW3 + j], v[(H2 > 0 ? VA2 : VA1) + j], o);
        float go = 0.0f;
        if (valid) {
          const float tt = __fmul_rn(small_int_to_float(ttg[r]), sig);
          const float ginv = __fdiv_rn(2.0f, (float)B);
          go = tus[r] ? __fmul_rn(__fsub_rn(o, tt), ginv) : 0.0f;
        }
        v[VGO] = go;
        v[VONE] = valid ? 1.0f : 0.0f;
      }
      __syncthreads();
      const float go = v[VGO];
      if constexpr (H2 > 0) {
#pragma unroll
        for (int jj = 0; jj < NU2; ++jj) {
          const int j = q * NU2 + jj;
          if (j < H2) {
            const float qq = __fmul_rn(go, w[OW3 + j]);
            v[VD2 + j] = valid ? (z2[jj] >= 0.0f ? qq : __fmul_rn(qq, kAlpha)) : 0.0f;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int jj = 0; jj < NU1; ++jj) {
        const int i = q * NU1 + jj;
        if (i < H1) {
          float d;
          if constexpr (H2 > 0) {
            float sacc = 0.0f;
#pragma unroll 8
            for (int j = 0; j < H2; ++j) sacc = __fmaf_rn(w[OW2 + j * H1 + i], v[VD2 + j], sacc);
            d = z1[jj] >= 0.0f ? sacc : __fmul_rn(sacc, kAlpha);
          } else {
            const float qq = __fmul_rn(go, w[OW3 + i]);
            d = z1[jj] >= 0.0f ? qq : __fmul_rn(qq, kAlpha);
          }
          v[VD1 + i] = valid ? d : 0.0f;
        }
      }
    }
    __syncthreads();
    // this CTA's 32-row sum of every parameter's terms, pairwise in row order
    for (int p = tid; p < NW; p += blockDim.x) {
      const int a = fa[p], b = fb[p];
      float t[kTrainRows];
#pragma unroll
      for (int r = 0; r < kTrainRows; ++r) t[r] = __fmul_rn(V[r * VS + a], V[r * VS + b]);
#pragma unroll
      for (int st = 1; st < kTrainRows; st <<= 1)
#pragma unroll
        for (int r = 0; r < kTrainRows; r += 2 * st) t[r] = __fadd_rn(t[r], t[r + st]);
      part[p] = t[0];
    }
    cl.sync();
    // the cluster sum of this CTA's slice, the update, and the new weights to every CTA
    for (int p = rank * SL + tid; p < NW && p < (rank + 1) * SL; p += blockDim.x) {
      float q[kTrainCluster];
#pragma unroll
      for (int c = 0; c < kTrainCluster; ++c) q[c] = peer_part[c][p];
      const float g = __fadd_rn(__fadd_rn(__fadd_rn(q[0], q[1]), __fadd_rn(q[2], q[3])),
                                __fadd_rn(__fadd_rn(q[4], q[5]), __fadd_rn(q[6], q[7])));
      const bool bias = (p >= OB1 && p < OB1 + H1) || (H2 > 0 && p >= OB2 && p < OB2 + H2) || p == NW - 1;
      float nv;
      if (bias) {
        nv = __fsub_rn(w[p], __fmul_rn(lr, g));
      } else {
        const float gt = __fadd_rn(g, __fmul_rn(lam2, w[p]));
        nv = __fsub_rn(w[p], __fmul_rn(lr, gt));
      }
#pragma unroll
      for (int c = 0; c < kTrainCluster; ++c) peer_w[c][p] = nv;
    }
    cl.sync();
  }
  if (rank == 0)
    for (int p = tid; p < NW; p += blockDim.x) wm[p] = w[p];
}

// validation cost; blockIdx.y = model (nmodels = Lorenzo)
template <int K, int H1, int H2>
__global__ void __launch_bounds__(256) k_val(const int* __restrict__ vin, const int* __restrict__ vtg,
                                             const uint8_t* __restrict__ vus, const float* __restrict__ wbuf,
                                             int nmodels, int m, const TrainCtl* __restrict__ ctl,
                                             unsigned long long* costs) {
  constexpr int NW = H1 * K + H1 + (H2 > 0 ? H2 * H1 + H2 : 0) + (H2 > 0 ? H2 : H1) + 1;
  __shared__ Mlp s_m;
  const int model = blockIdx.y;
  const bool lz = model == nmodels;
  if (!lz)
    for (int p = threadIdx.x; p < NW; p += blockDim.x) s_m.w[p] = wbuf[(size_t)model * NW + p];
  if (threadIdx.x == 0) { s_m.k = K; s_m.h1 = H1; s_m.h2 = H2; s_m.s_in = ctl->s_in; }
  __syncthreads();
  const int s_in = ctl->s_in;
  const float sig = __uint_as_float((unsigned int)(127 - s_in) << 23);
  const float unsig = __uint_as_float((unsigned int)(127 + s_in) << 23);
  const long long R = 1ll << (m - 1);
  const unsigned long long n = ctl->nval;
  unsigned long long cost = 0;
  auto bits = [&](unsigned long long i, long long pr) {
    const long long d = (long long)vtg[i] - pr;
    const unsigned long long a = (unsigned long long)(d < 0 ? -d : d);
    return (unsigned long long)bitlen_u((unsigned int)(a < (unsigned long long)R ? a : (unsigned long long)R));
  };
  // two samples per thread: the packed forward gives each the scalar forward's bits
  for (unsigned long long i2 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; 2 * i2 < n;
       i2 += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long i0 = 2 * i2, i1 = i0 + 1;
    const bool u0 = vus[i0] != 0, u1 = i1 < n && vus[i1] != 0;
    if (!u0 && !u1) continue;
    int in0[K], in1[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      in0[q] = vin[i0 * K + q];
      in1[q] = i1 < n ? vin[i1 * K + q] : 0;
    }
    long long p0 = 0, p1 = 0;
    if (lz) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        p0 += (long long)lz_w(K, q) * in0[q];
        p1 += (long long)lz_w(K, q) * in1[q];
      }
    } else {
      float f0, f1;
      mlp_fwd2<K, H1, H2>(s_m, in0, in1, sig, unsig, f0, f1);
      p0 = round_pred(f0);
      p1 = round_pred(f1);
    }
    if (u0) cost += bits(i0, p0);
    if (u1) cost += bits(i1, p1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cost += __shfl_xor_sync(0xFFFFFFFFu, cost, o);
  if ((threadIdx.x & 31) == 0 && cost) atomicAdd(&costs[model], cost);
}

__global__ void k_choose(const unsigned long long* costs, int nmodels, TrainCtl* ctl) {
  unsigned long long best = costs[nmodels];
  int bi = -1;
  for (int h = 0; h < nmodels; ++h)
    if (costs[h] < best) { best = costs[h]; bi = h; }
  ctl->chosen = bi;
}

template <int K, int H1, int H2>
static int launch_train_models(const TrainBufs& tb, int nmodels, int m, cudaStream_t s) {
  {
    ProfScope p(kStTrain, s);
    k_train<K, H1, H2><<<nmodels * kTrainCluster, 32 * kTrainWarps, 0, s>>>(
        tb.tin, tb.ttg, tb.tus, tb.w, tb.lrs, tb.lams, reinterpret_cast<const TrainCtl*>(tb.ctl));
  }
  dim3 gv(152, nmodels + 1);
  k_val<K, H1, H2><<<gv, 256, 0, s>>>(tb.vin, tb.vtg, tb.vus, tb.w, nmodels, m,
                                      reinterpret_cast<const TrainCtl*>(tb.ctl), tb.costs);
  k_choose<<<1, 1, 0, s>>>(tb.costs, nmodels, reinterpret_cast<TrainCtl*>(tb.ctl));
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Selection by simulated compression (Section IV.C).  k_valhist quantizes
// every model's (blockIdx.y; nmodels = Lorenzo) validation residuals as the
// compressor would (code k + R, or 0 for a balance point) into its histogram
// and counts residual bit lengths for the coverage rule; the codebook kernel
// then builds each histogram's Huffman lengths, and k_simsize adds up the
// coded bits plus the stored value of every balance point.
// ---------------------------------------------------------------------------
template <int K, int H1, int H2>
__global__ void __launch_bounds__(256) k_valhist(const int* __restrict__ vin, const int* __restrict__ vtg,
                                                 const uint8_t* __restrict__ vus, const float* __restrict__ wbuf,
                                                 int nmodels, int m, const TrainCtl* __restrict__ ctl,
                                                 unsigned long long* hists, unsigned long long* bitcnt) {
  constexpr int NW = H1 * K + H1 + (H2 > 0 ? H2 * H1 + H2 : 0) + (H2 > 0 ? H2 : H1) + 1;
  __shared__ Mlp s_m;
  __shared__ unsigned int s_bc[34];
  const int model = blockIdx.y;
  const bool lz = model == nmodels;
  if (!lz)
    for (int p = threadIdx.x; p < NW; p += blockDim.x) s_m.w[p] = wbuf[(size_t)model * NW + p];
  if (threadIdx.x == 0) { s_m.k = K; s_m.h1 = H1; s_m.h2 = H2; s_m.s_in = ctl->s_in; }
  if (threadIdx.x < 34) s_bc[threadIdx.x] = 0u;
  __syncthreads();
  const int s_in = ctl->s_in;
  const float sig = __uint_as_float((unsigned int)(127 - s_in) << 23);
  const float unsig = __uint_as_float((unsigned int)(127 + s_in) << 23);
  const long long R = 1ll << (m - 1);
  const unsigned long long n = ctl->nval;
  unsigned long long* hist = hists + ((size_t)model << m);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    if (!vus[i]) continue;
    int in[K];
#pragma unroll
    for (int q = 0; q < K; ++q) in[q] = vin[i * K + q];
    long long pr = 0;
    if (lz) {
#pragma unroll
      for (int q = 0; q < K; ++q) pr += (long long)lz_w(K, q) * in[q];
    } else {
      pr = round_pred(mlp_fwd<K, H1, H2>(s_m, in, sig, unsig));
    }
    const long long d = (long long)vtg[i] - pr;
    const unsigned long long a = (unsigned long long)(d < 0 ? -d : d);
    atomicAdd(&hist[a <= (unsigned long long)(R - 1) ? (unsigned int)(d + R) : 0u], 1ull);
    atomicAdd(&s_bc[64 - __clzll((long long)a)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 34 && s_bc[threadIdx.x])
    atomicAdd(&bitcnt[(size_t)model * 34 + threadIdx.x], (unsigned long long)s_bc[threadIdx.x]);
}

// Coded bits of one histogram from its codebook list (sym | len << 16, n_used
// entries), plus value_bits per balance point (symbol 0).
__global__ void __launch_bounds__(256) k_simsize(const unsigned long long* __restrict__ hist,
                                                 const uint8_t* __restrict__ list, const State* __restrict__ st,
                                                 int value_bits, unsigned long long* size_out) {
  __shared__ unsigned long long s_part[8];
  const unsigned int n = st->err ? 0u : st->n_used;
  unsigned long long acc = 0;
  for (unsigned int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned int e = reinterpret_cast<const unsigned int*>(list)[i];
    acc += hist[e & 0xFFFFu] * (unsigned long long)(e >> 16);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = hist[0] * (unsigned long long)value_bits;
    for (int w = 0; w < 8; ++w) t += s_part[w];
    *size_out = t;
  }
}

template <int K, int H1, int H2>
static int launch_select_models(const TrainBufs& tb, const SelectBufs& sb, int nmodels, int m, int value_bits,
                                cudaStream_t s) {
  const size_t nsym = (size_t)1 << m;
  if (cudaMemsetAsync(sb.hists, 0, 8 * nsym * (nmodels + 1), s) != cudaSuccess ||
      cudaMemsetAsync(sb.bitcnt, 0, 8 * 34 * (size_t)(nmodels + 1), s) != cudaSuccess)
    return PC_ERR_CUDA;
  dim3 gv(152, nmodels + 1);
  k_valhist<K, H1, H2><<<gv, 256, 0, s>>>(tb.vin, tb.vtg, tb.vus, tb.w, nmodels, m,
                                          reinterpret_cast<const TrainCtl*>(tb.ctl), sb.hists, sb.bitcnt);
  if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  for (int h = 0; h <= nmodels; ++h) {
    if (cudaMemsetAsync(sb.st, 0, sizeof(State), s) != cudaSuccess) return PC_ERR_CUDA;
    int r = launch_huff_list(sb.hists + (h << m), m, sb.st, sb.hs, sb.list, 4 * nsym + 64, s);
    if (r) return r;
    k_simsize<<<1, 256, 0, s>>>(sb.hists + (h << m), sb.list, sb.st, value_bits, tb.costs + h);
  }
  k_choose<<<1, 1, 0, s>>>(tb.costs, nmodels, reinterpret_cast<TrainCtl*>(tb.ctl));
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

int launch_select(const TrainBufs& tb, const SelectBufs& sb, int k, int h1, int h2, int m, int nmodels,
                  int value_bits, cudaStream_t s) {
  if (cudaMemsetAsync(tb.costs, 0, sizeof(unsigned long long) * (nmodels + 1), s) != cudaSuccess) return PC_ERR_CUDA;
#define PC_SEL(KK, A, B) \
  if (k == KK && h1 == A && h2 == B) return launch_select_models<KK, A, B>(tb, sb, nmodels, m, value_bits, s);
  PC_SEL(7, 16, 16)
  PC_SEL(13, 32, 32)
  PC_SEL(7, 8, 8)
  PC_SEL(7, 2, 0)
  PC_SEL(13, 16, 16)
#undef PC_SEL
  return PC_ERR_ARG;
}

// ---------------------------------------------------------------------------
// Sample codebook (Section IV.C): the validation samples of the training
// phase (seed, thr32), their residuals under the given FP32 weights (model 0)
// or Lorenzo quantized into a histogram at m code bits, symbol 0 counted at
// least once, and its Huffman code as a codebook list in sb.list (n_used in
// sb.st).
// ---------------------------------------------------------------------------
__global__ void k_set_sin(TrainCtl* ctl, int s_in) { ctl->s_in = s_in; }
// Symbol 0 counts at least once; with span_fill every code between the
// smallest and the largest sampled code (symbols >= 1) counts at least once.
__global__ void __launch_bounds__(1024) k_sample_fill(unsigned long long* hist, int nsym, int span_fill) {
  __shared__ int s_lo, s_hi;
  if (threadIdx.x == 0) {
    s_lo = nsym;
    s_hi = 0;
  }
  __syncthreads();
  if (span_fill) {
    int lo = nsym, hi = 0;
    for (int c = 1 + threadIdx.x; c < nsym; c += blockDim.x)
      if (hist[c]) {
        lo = min(lo, c);
        hi = max(hi, c);
      }
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
    __syncthreads();
    for (int c = s_lo + threadIdx.x; c <= s_hi; c += blockDim.x)
      if (hist[c] == 0ull) hist[c] = 1ull;
  }
  if (threadIdx.x == 0 && hist[0] == 0ull) hist[0] = 1ull;
}

template <int K, int H1, int H2>
static int launch_sample_hist_k(const TrainBufs& tb, const SelectBufs& sb, int m, bool lorenzo, int span_fill,
                                cudaStream_t s) {
  const size_t nsym = (size_t)1 << m;
  if (cudaMemsetAsync(sb.hists, 0, 8 * nsym * 2, s) != cudaSuccess ||
      cudaMemsetAsync(sb.bitcnt, 0, 8 * 34 * 2, s) != cudaSuccess)
    return PC_ERR_CUDA;
  dim3 gv(152, 2);
  k_valhist<K, H1, H2><<<gv, 256, 0, s>>>(tb.vin, tb.vtg, tb.vus, tb.w, 1, m,
                                          reinterpret_cast<const TrainCtl*>(tb.ctl), sb.hists, sb.bitcnt);
  unsigned long long* h = sb.hists + (lorenzo ? nsym : 0);
  k_sample_fill<<<1, 1024, 0, s>>>(h, (int)nsym, span_fill);
  if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  if (cudaMemsetAsync(sb.st, 0, sizeof(State), s) != cudaSuccess) return PC_ERR_CUDA;
  return launch_huff_list(h, m, sb.st, sb.hs, sb.list, 4 * nsym + 64, s);
}

template <typename T>
int launch_sample_hist(const T* x, const Geo& g, const State* st, const Tabs* tabs, const TrainBufs& tb,
                       const SelectBufs& sb, int k, int h1, int h2, int s_in, int m, bool lorenzo, int span_fill,
                       unsigned long long seed, unsigned int thr32, cudaStream_t s) {
  TrainCtl* ctl = reinterpret_cast<TrainCtl*>(tb.ctl);
  if (cudaMemsetAsync(ctl, 0, sizeof(TrainCtl), s) != cudaSuccess) return PC_ERR_CUDA;
  const unsigned int nb8 = (unsigned int)((g.nblocks + 7) / 8);
  k_samp_count<<<nb8, 256, 0, s>>>(g, seed, thr32, tb.cnt_t, tb.cnt_v);
  k_samp_scan<<<1, 1024, 0, s>>>(g.nblocks, tb.cnt_t, tb.cnt_v, tb.off_t, tb.off_v, ctl);
  const size_t gsm = sizeof(Tabs) + 4ull * g.bvol * 4;
  if (cudaFuncSetAttribute(k_samp_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm) != cudaSuccess)
    return PC_ERR_CUDA;
  k_samp_gather<T><<<(unsigned int)((g.nblocks + 3) / 4), 128, gsm, s>>>(
      x, g, st, tabs, seed, thr32, k, tb.off_t, tb.off_v, tb.tin, tb.ttg, tb.tus, tb.vin, tb.vtg, tb.vus, ctl,
      tb.cap_t, tb.cap_v);
  k_set_sin<<<1, 1, 0, s>>>(ctl, s_in);
  if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  if (lorenzo) return launch_sample_hist_k<7, 16, 16>(tb, sb, m, true, span_fill, s);
  if (k == 7 && h1 == 16 && h2 == 16) return launch_sample_hist_k<7, 16, 16>(tb, sb, m, false, span_fill, s);
  if (k == 13 && h1 == 32 && h2 == 32) return launch_sample_hist_k<13, 32, 32>(tb, sb, m, false, span_fill, s);
  if (k == 7 && h1 == 8 && h2 == 8) return launch_sample_hist_k<7, 8, 8>(tb, sb, m, false, span_fill, s);
  if (k == 7 && h1 == 2 && h2 == 0) return launch_sample_hist_k<7, 2, 0>(tb, sb, m, false, span_fill, s);
  if (k == 13 && h1 == 16 && h2 == 16) return launch_sample_hist_k<13, 16, 16>(tb, sb, m, false, span_fill, s);
  return PC_ERR_ARG;
}
template int launch_sample_hist<float>(const float*, const Geo&, const State*, const Tabs*, const TrainBufs&,
                                       const SelectBufs&, int, int, int, int, int, bool, int, unsigned long long,
                                       unsigned int, cudaStream_t);
template int launch_sample_hist<double>(const double*, const Geo&, const State*, const Tabs*, const TrainBufs&,
                                        const SelectBufs&, int, int, int, int, int, bool, int, unsigned long long,
                                        unsigned int, cudaStream_t);

size_t train_ctl_bytes() { return sizeof(TrainCtl); }

template <typename T>
int launch_train(const T* x, const Geo& g, const State* st, const Tabs* tabs, const TrainBufs& tb, int k, int h1,
                 int h2, int m, int nmodels, unsigned long long seed, unsigned int thr32, cudaStream_t s) {
  TrainCtl* ctl = reinterpret_cast<TrainCtl*>(tb.ctl);
  if (cudaMemsetAsync(ctl, 0, sizeof(TrainCtl), s) != cudaSuccess) return PC_ERR_CUDA;
  if (cudaMemsetAsync(tb.costs, 0, sizeof(unsigned long long) * (nmodels + 1), s) != cudaSuccess) return PC_ERR_CUDA;
  const unsigned int nb8 = (unsigned int)((g.nblocks + 7) / 8);
  k_samp_count<<<nb8, 256, 0, s>>>(g, seed, thr32, tb.cnt_t, tb.cnt_v);
  k_samp_scan<<<1, 1024, 0, s>>>(g.nblocks, tb.cnt_t, tb.cnt_v, tb.off_t, tb.off_v, ctl);
  const size_t gsm = sizeof(Tabs) + 4ull * g.bvol * 4;
  if (cudaFuncSetAttribute(k_samp_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm) != cudaSuccess)
    return PC_ERR_CUDA;
  k_samp_gather<T><<<(unsigned int)((g.nblocks + 3) / 4), 128, gsm, s>>>(
      x, g, st, tabs, seed, thr32, k, tb.off_t, tb.off_v, tb.tin, tb.ttg, tb.tus, tb.vin, tb.vtg, tb.vus, ctl,
      tb.cap_t, tb.cap_v);
  k_in_shift<<<304, 256, 0, s>>>(tb.ttg, tb.tus, ctl);
  const int nw = h1 * k + h1 + (h2 > 0 ? h2 * h1 + h2 : 0) + (h2 > 0 ? h2 : h1) + 1;
  k_init_w<<<(nw + 255) / 256, 256, 0, s>>>(tb.w, nmodels, k, h1, h2, seed ^ 0x5DEECE66Dull, ctl);
  if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  if (k == 7 && h1 == 16 && h2 == 16) return launch_train_models<7, 16, 16>(tb, nmodels, m, s);
  if (k == 13 && h1 == 32 && h2 == 32) return launch_train_models<13, 32, 32>(tb, nmodels, m, s);
  if (k == 7 && h1 == 8 && h2 == 8) return launch_train_models<7, 8, 8>(tb, nmodels, m, s);
  if (k == 7 && h1 == 2 && h2 == 0) return launch_train_models<7, 2, 0>(tb, nmodels, m, s);
  if (k == 13 && h1 == 16 && h2 == 16) return launch_train_models<13, 16, 16>(tb, nmodels, m, s);
  return PC_ERR_ARG;
}
// ---------------------------------------------------------------------------
// Fixed-point (BF16) form of a trained perceptron.  Weights of layer l become
// integers |Wq| <= 255 times 2^-e_l, with e_l the largest exponent such that
// max|W_l| 2^e_l <= 255 (kept in [-30, 30]); biases become integers in the
// units of their layer's sums (clamped to +-2^30); each hidden layer's shift
// t is the smallest t in [0, 40] with max 16 |leaky(A)| 2^-t <= 16 (2^15 - 1)
// over the used training and validation samples.
// ---------------------------------------------------------------------------
__device__ int q_wexp(float m) {
  if (m == 0.0f) return 0;
  int E;
  const float fr = frexpf(m, &E);
  const int e = fr <= 255.0f / 256.0f ? 8 - E : 7 - E;
  return e < -30 ? -30 : (e > 30 ? 30 : e);
}
__device__ long long q_w(float w, int e) { return (long long)rintf(ldexpf(w, e)); }
__device__ long long q_b(float b, int E) {
  const double v = rint(ldexp((double)b, E));
  const double lim = 1073741824.0;  // 2^30
  return (long long)(v > lim ? lim : (v < -lim ? -lim : v));
}

// one CTA: exponents, integer weights, layer-1 biases, header of the network
__global__ void __launch_bounds__(256) k_qweights(const float* __restrict__ w, int k, int h1, int h2, const TrainCtl* ctl,
                                                  long long* q, unsigned long long* qmax) {
  __shared__ unsigned int s_m[3];
  const int tid = threadIdx.x;
  if (tid < 3) s_m[tid] = 0u;
  __syncthreads();
  const float* W1 = w;
  const float* W2 = W1 + h1 * k + h1;
  const float* W3 = W2 + h2 * h1 + h2;
  for (int i = tid; i < h1 * k; i += 256) atomicMax(&s_m[0], __float_as_uint(fabsf(W1[i])));
  for (int i = tid; i < h2 * h1; i += 256) atomicMax(&s_m[1], __float_as_uint(fabsf(W2[i])));
  for (int i = tid; i < h2; i += 256) atomicMax(&s_m[2], __float_as_uint(fabsf(W3[i])));
  __syncthreads();
  const int s_in = ctl->s_in;
  const int e1 = q_wexp(__uint_as_float(s_m[0])), e2 = q_wexp(__uint_as_float(s_m[1])),
            e3 = q_wexp(__uint_as_float(s_m[2]));
  long long* QW1 = q + kQHdr;
  long long* QB1 = QW1 + h1 * k;
  long long* QW2 = QB1 + h1;
  long long* QW3 = QW2 + h2 * h1 + h2;
  for (int i = tid; i < h1 * k; i += 256) QW1[i] = q_w(W1[i], e1);
  for (int i = tid; i < h1; i += 256) QB1[i] = q_b(W1[h1 * k + i], e1 + s_in);
  for (int i = tid; i < h2 * h1; i += 256) QW2[i] = q_w(W2[i], e2);
  for (int i = tid; i < h2; i += 256) QW3[i] = q_w(W3[i], e3);
  if (tid == 0) {
    q[0] = k; q[1] = h1; q[2] = h2; q[3] = s_in;
    q[4] = e1; q[5] = e2; q[6] = e3; q[7] = 0; q[8] = 0;
    qmax[0] = 0ull;
    qmax[1] = 0ull;
  }
}

// max 16 |leaky(A)| of hidden layer L (1 or 2) over the used samples
template <int L>
__global__ void __launch_bounds__(256) k_qscan(const int* __restrict__ tin, const uint8_t* __restrict__ tus,
                                               const int* __restrict__ vin, const uint8_t* __restrict__ vus,
                                               const TrainCtl* ctl, const long long* __restrict__ q,
                                               unsigned long long* qmax) {
  const int k = (int)q[0], h1 = (int)q[1], h2 = (int)q[2], t1 = (int)q[7];
  const long long* W1 = q + kQHdr;
  const long long* B1 = W1 + h1 * k;
  const long long* W2 = B1 + h1;
  const long long* B2 = W2 + h2 * h1;
  const unsigned long long nt = ctl->ntrain, nv = ctl->nval;
  unsigned long long m = 0;
  for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < nt + nv; i += gridDim.x * 256ull) {
    const bool isv = i >= nt;
    const unsigned long long si = isv ? i - nt : i;
    if (!(isv ? vus[si] : tus[si])) continue;
    const int* in = (isv ? vin : tin) + si * (unsigned long long)k;
    int x[13];
    for (int c = 0; c < k; ++c) x[c] = in[c] > kQIn ? kQIn : (in[c] < -kQIn ? -kQIn : in[c]);
    int h1q[kMaxH];
    for (int j = 0; j < h1; ++j) {
      int acc = 0;
      for (int c = 0; c < k; ++c) acc += (int)W1[j * k + c] * x[c];
      const long long a = (long long)acc + B1[j];
      if (L == 1) {
        const unsigned long long l16 = (unsigned long long)(a >= 0 ? 16 * a : -a);
        m = l16 > m ? l16 : m;
      } else {
        h1q[j] = leaky_requant32((int)a, t1, (1 << t1) >> 1, (1 << (t1 + 4)) >> 1);
      }
    }
    if (L == 2) {
      for (int j = 0; j < h2; ++j) {
        int acc = 0;
        for (int c = 0; c < h1; ++c) acc += (int)W2[j * h1 + c] * h1q[c];
        const long long a = (long long)acc + B2[j];
        const unsigned long long l16 = (unsigned long long)(a >= 0 ? 16 * a : -a);
        m = l16 > m ? l16 : m;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&qmax[L - 1], m);
}

// shift of hidden layer L from its maximum; then the next layer's biases
template <int L>
__global__ void k_qshift(const float* __restrict__ w, long long* q, const unsigned long long* qmax) {
  if (threadIdx.x != 0) return;
  const int k = (int)q[0], h1 = (int)q[1], h2 = (int)q[2], s_in = (int)q[3];
  const int e1 = (int)q[4], e2 = (int)q[5], e3 = (int)q[6];
  const unsigned long long M = qmax[L - 1];
  const unsigned long long lim = 16ull * (unsigned long long)kQAct;
  int t = 40;
  for (int c = 0; c < 40; ++c)
    if (M <= (lim << c)) { t = c; break; }
  const float* b2 = w + h1 * k + h1 + h2 * h1;
  const float* b3 = b2 + h2 + h2;
  long long* QB2 = q + kQHdr + h1 * k + h1 + h2 * h1;
  long long* QB3 = QB2 + h2 + h2;
  if (L == 1) {
    q[7] = t;
    for (int j = 0; j < h2; ++j) QB2[j] = q_b(b2[j], e1 + e2 + s_in - t);
  } else {
    q[8] = t;
    QB3[0] = q_b(b3[0], e1 + e2 + e3 + s_in - (int)q[7] - t);
  }
}

template <typename T>
int launch_quantize(const T* x, const Geo& g, const State* st, const Tabs* tabs, const TrainBufs& tb, int k, int h1,
                    int h2, int s_in, unsigned long long seed, unsigned int thr32, long long* q,
                    unsigned long long* qmax, cudaStream_t s) {
  TrainCtl* ctl = reinterpret_cast<TrainCtl*>(tb.ctl);
  if (cudaMemsetAsync(ctl, 0, sizeof(TrainCtl), s) != cudaSuccess) return PC_ERR_CUDA;
  const unsigned int nb8 = (unsigned int)((g.nblocks + 7) / 8);
  k_samp_count<<<nb8, 256, 0, s>>>(g, seed, thr32, tb.cnt_t, tb.cnt_v);
  k_samp_scan<<<1, 1024, 0, s>>>(g.nblocks, tb.cnt_t, tb.cnt_v, tb.off_t, tb.off_v, ctl);
  const size_t gsm = sizeof(Tabs) + 4ull * g.bvol * 4;
  if (cudaFuncSetAttribute(k_samp_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm) != cudaSuccess)
    return PC_ERR_CUDA;
  k_samp_gather<T><<<(unsigned int)((g.nblocks + 3) / 4), 128, gsm, s>>>(
      x, g, st, tabs, seed, thr32, k, tb.off_t, tb.off_v, tb.tin, tb.ttg, tb.tus, tb.vin, tb.vtg, tb.vus, ctl,
      tb.cap_t, tb.cap_v);
  // the input scale is the caller's (the one the weights were trained with)
  if (cudaMemcpyAsync(&ctl->s_in, &s_in, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) return PC_ERR_CUDA;
  k_qweights<<<1, 256, 0, s>>>(tb.w, k, h1, h2, ctl, q, qmax);
  k_qscan<1><<<304, 256, 0, s>>>(tb.tin, tb.tus, tb.vin, tb.vus, ctl, q, qmax);
  k_qshift<1><<<1, 32, 0, s>>>(tb.w, q, qmax);
  k_qscan<2><<<304, 256, 0, s>>>(tb.tin, tb.tus, tb.vin, tb.vus, ctl, q, qmax);
  k_qshift<2><<<1, 32, 0, s>>>(tb.w, q, qmax);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
template int launch_quantize<float>(const float*, const Geo&, const State*, const Tabs*, const TrainBufs&, int, int,
                                    int, int, unsigned long long, unsigned int, long long*, unsigned long long*,
                                    cudaStream_t);
template int launch_quantize<double>(const double*, const Geo&, const State*, const Tabs*, const TrainBufs&, int, int,
                                     int, int, unsigned long long, unsigned int, long long*, unsigned long long*,
                                     cudaStream_t);

template int launch_train<float>(const float*, const Geo&, const State*, const Tabs*, const TrainBufs&, int, int, int,
                                 int, int, unsigned long long, unsigned int, cudaStream_t);
template int launch_train<double>(const double*, const Geo&, const State*, const Tabs*, const TrainBufs&, int, int,
                                  int, int, int, unsigned long long, unsigned int, cudaStream_t);

}  // namespace pc
