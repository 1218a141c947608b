// Compression kernels: statistics (a1), constants (a2), and the fused
// transform / predict / select / quantize / histogram pass (a4-a9).
#include "pc_kernels.cuh"
#include "pc_qmlp.cuh"
#include "pc_tcnet.cuh"
#include "pc_profile.cuh"

namespace pc {

// ---------------------------------------------------------------------------
// a0: reset the per-call state and the histogram.
// ---------------------------------------------------------------------------
__global__ void k_init(State* st, unsigned long long* hist, int nsym) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    State z;
    memset(&z, 0, sizeof(z));
    z.amin_bits = ~0ull;
    *st = z;
  }
  for (; i < nsym; i += gridDim.x * blockDim.x) hist[i] = 0ull;
}

// ---------------------------------------------------------------------------
// a1: abs_min over normal magnitudes, abs_max over all, non-finite flag
// (Algorithm 1 input; Section III.B defines min as the non-zero minimum
// absolute value).  Magnitude bit patterns order like unsigned integers, so
// the reduction is exact and order-free.
// ---------------------------------------------------------------------------
template <typename T> struct Bits;
template <> struct Bits<float> {
  using U = unsigned int;
  static __device__ __forceinline__ U mag(float v) { return __float_as_uint(v) & 0x7FFFFFFFu; }
  static constexpr U kInf = 0x7F800000u, kMinNormal = 0x00800000u;
};
template <> struct Bits<double> {
  using U = unsigned long long;
  static __device__ __forceinline__ U mag(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  }
  static constexpr U kInf = 0x7FF0000000000000ull, kMinNormal = 0x0010000000000000ull;
};

template <typename T>
__global__ void __launch_bounds__(256) k_stats(const T* __restrict__ x, unsigned long long n, State* st) {
  using B = Bits<T>;
  using U = typename B::U;
  // in the value's own width: the largest magnitude (non-finite ones sort
  // above every finite one) and the smallest normal magnitude (the all-ones
  // start means none)
  U mn = ~U(0), mx = 0;
  auto acc = [&](T v) {
    const U a = B::mag(v);
    mx = max(mx, a);
    mn = min(mn, (a >= B::kMinNormal && a < B::kInf) ? a : ~U(0));
  };
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long tid0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  // 16-byte vector loads over the aligned body, four in flight per thread;
  // scalar loads for the tail
  constexpr int V = 16 / sizeof(T);
  constexpr int NL = 4;
  const bool aligned = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
  const unsigned long long nv = aligned ? n / V : 0;
  const uint4* xv = reinterpret_cast<const uint4*>(x);
  unsigned long long i = tid0;
  for (; i + (NL - 1) * stride < nv; i += NL * stride) {
    uint4 u[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) u[k] = __ldg(&xv[i + k * stride]);
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      T t[V];
      memcpy(t, &u[k], 16);
#pragma unroll
      for (int q = 0; q < V; ++q) acc(t[q]);
    }
  }
  for (; i < nv; i += stride) {
    const uint4 u = __ldg(&xv[i]);
    T t[V];
    memcpy(t, &u, 16);
#pragma unroll
    for (int q = 0; q < V; ++q) acc(t[q]);
  }
  for (unsigned long long j = nv * V + tid0; j < n; j += stride) acc(__ldg(&x[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, (U)__shfl_xor_sync(0xFFFFFFFFu, mn, o));
    mx = max(mx, (U)__shfl_xor_sync(0xFFFFFFFFu, mx, o));
  }
  __shared__ U s_mn[8], s_mx[8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { s_mn[w] = mn; s_mx[w] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      mn = min(mn, s_mn[k]);
      mx = max(mx, s_mx[k]);
    }
    const bool have = mn != ~U(0);
    if (have) atomicMin(&st->amin_bits, (unsigned long long)mn);
    atomicMax(&st->amax_bits, (unsigned long long)mx);
    if (mx >= B::kInf) atomicOr(&st->nonfinite, 1u);
    if (have) atomicOr(&st->have_normal, 1u);
  }
}

// ---------------------------------------------------------------------------
// a2: constants (Eq. 8-12), one thread, double precision:
//   b_a = log2(1 + eb), step = 2 b_a;
//   Kp = rint(log2 abs_min / step)                       (factor_pos = abs_min)
//   log2 factor_neg = log2(abs_max + e0) + log2 abs_min + step - log2(abs_min - e0)
//   Kn = rint(log2 factor_neg / step)
//   Zq = rint(log2 e0 / step) + Kp                       (zero image, Eq. 12)
//   S  = rint(log2(abs_max + e0) / step) + Kp            (sign boundary)
// with e0 the smallest positive value of the dtype.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_consts(State* st, double eb, Tabs* tabs) {
  // four independent logarithms on four threads, combined by thread 0
  // (launched with 128 threads, one per log/reciprocal table entry)
  __shared__ double s_l[4];
  __shared__ double s_ab[2];
  __shared__ int s_stop;
  State& c = *st;
  constexpr bool f32 = sizeof(T) == 4;
  const double e0 = f32 ? 0x1p-149 : 0x1p-1074;
  const int t = threadIdx.x;
  if (t == 0) {
    s_stop = 0;
    if (c.nonfinite) {
      c.err = PC_ERR_NONFINITE;
      s_stop = 1;
    }
    double amin, amax;
    if (c.have_normal) {
      if (f32) {
        amin = (double)__uint_as_float((unsigned int)c.amin_bits);
        amax = (double)__uint_as_float((unsigned int)c.amax_bits);
      } else {
        amin = __longlong_as_double((long long)c.amin_bits);
        amax = __longlong_as_double((long long)c.amax_bits);
      }
      c.trivial = 0;
    } else {
      amin = 1.0; amax = 1.0; c.trivial = 1;
    }
    c.amin = amin;
    c.amax = amax;
    s_ab[0] = amin;
    s_ab[1] = amax;
  }
  __syncthreads();
  if (s_stop) return;
  build_tabs_entry(tabs, t);  // one table entry per thread (128 threads: four warps share the FP64 work)
  if (t < 4) {
    const double amin = s_ab[0], amax = s_ab[1];
    const double arg = t == 0 ? __dadd_rn(1.0, eb) : (t == 1 ? __dadd_rn(amax, e0) : (t == 2 ? amin : __dsub_rn(amin, e0)));
    s_l[t] = dev_log2d(arg);
  }
  __syncthreads();
  if (t != 0) return;
  const double le0 = f32 ? -149.0 : -1074.0;
  const double ba = s_l[0];
  const double step = __dadd_rn(ba, ba);
  const double lmax = s_l[1], lmin = s_l[2];
  double kp = rint(__ddiv_rn(lmin, step));
  double lfn = __dsub_rn(__dadd_rn(__dadd_rn(lmax, lmin), step), s_l[3]);
  double kn = rint(__ddiv_rn(lfn, step));
  double zq = __dadd_rn(rint(__ddiv_rn(le0, step)), kp);
  double s = __dadd_rn(rint(__ddiv_rn(lmax, step)), kp);
  double span = __dadd_rn(__ddiv_rn(f32 ? 151.0 : 1076.0, step), 2.0);
  const double lim = 1073741824.0;
  if (__dadd_rn(fabs(kp), span) > lim || __dadd_rn(fabs(kn), span) > lim || fabs(zq) > lim || fabs(s) > lim) {
    c.err = PC_ERR_EB_RANGE;
    return;
  }
  c.Kp = (int)kp; c.Kn = (int)kn; c.Zq = (int)zq; c.S = (int)s;
  c.step32 = __double2float_rn(step);
  c.inv32 = __fdiv_rn(1.0f, c.step32);
  float ef = __double2float_rn(eb);
  if ((double)ef > eb) ef = nextafterf(ef, 0.0f);
  c.ebdn32 = ef;
  c.stepd = step;
  c.invd = __ddiv_rn(1.0, step);
  c.ebdnd = eb;
}

// ---------------------------------------------------------------------------
// a4-a9: fused transform, prediction, block select, quantization, histogram.
//
// A CTA of 256 threads handles a brick of G consecutive blocks along x (G
// chosen so a brick holds at most 4096 points); each block is owned by a team
// of 256/G threads.  The brick is read with consecutive threads on consecutive
// x (16-byte loads when rows allow), transformed on the fly and kept on chip:
// each point's code with its bound flag (2 q + ok), and the clamped
// anchor-centred inputs in a zero-bordered padded block, so that stencil
// gathers need no bounds checks (a neighbour outside the block reads 0).
// Codes go out block-strided in padded raster order (index (lz*B1 + ly)*B2 +
// lx) with 16-byte stores; the histogram is kept in shared memory for a
// window of codes around R and flushed once per CTA.
// ---------------------------------------------------------------------------
constexpr int kHistWin = 2048;

// Exclusive scan of two counters over the TS threads of a team (TS = 32 or a
// multiple of 32 that divides 256); ta, tb receive the team totals.  For
// TS > 32 it synchronizes the CTA (all teams call it together).
template <int TS>
__device__ __forceinline__ void team_exscan2(unsigned int a, unsigned int b, unsigned int& pa, unsigned int& pb,
                                             unsigned int& ta, unsigned int& tb, unsigned int* s_scr) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned int xa = a, xb = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int ya = __shfl_up_sync(0xFFFFFFFFu, xa, o);
    const unsigned int yb = __shfl_up_sync(0xFFFFFFFFu, xb, o);
    if (lane >= o) { xa += ya; xb += yb; }
  }
  if constexpr (TS == 32) {
    pa = xa - a;
    pb = xb - b;
    ta = __shfl_sync(0xFFFFFFFFu, xa, 31);
    tb = __shfl_sync(0xFFFFFFFFu, xb, 31);
  } else {
    constexpr int NW = TS / 32;
    if (lane == 31) { s_scr[w] = xa; s_scr[8 + w] = xb; }
    __syncthreads();
    const int w0 = (w / NW) * NW;
    unsigned int oa = 0, ob = 0, sa = 0, sb = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      const unsigned int va = s_scr[w0 + i], vb = s_scr[8 + w0 + i];
      if (w0 + i < w) { oa += va; ob += vb; }
      sa += va;
      sb += vb;
    }
    pa = oa + xa - a;
    pb = ob + xb - b;
    ta = sa;
    tb = sb;
    __syncthreads();
  }
}

// Decoupled look-back over the bricks of a field (one warp): publish this
// brick's aggregate, add up the aggregates of the bricks before it back to
// the nearest published inclusive prefix, publish this brick's inclusive
// prefix and return its exclusive one.  Records are flag << 62 | value with
// flag 1 = aggregate, 2 = inclusive prefix (0: not yet written).  Bricks are
// handed out in order to running CTAs and a brick publishes its aggregate
// before it waits, so every wait ends; it is still bounded, and a wait that
// runs out sets PC_ERR_TIMEOUT and takes the sum so far.
constexpr unsigned int kLookbackPolls = 1u << 21;
__device__ __forceinline__ unsigned long long lookback(unsigned long long* rec, long long k, unsigned long long agg,
                                                       int lane, int* errw) {
  constexpr unsigned long long kA = 1ull << 62, kP = 2ull << 62, kV = (1ull << 62) - 1;
  volatile unsigned long long* vr = rec;
  if (k == 0) {
    if (lane == 0) vr[0] = kP | agg;
    return 0ull;
  }
  if (lane == 0) vr[k] = kA | agg;
  unsigned long long excl = 0;
  long long base = k - 1;
  unsigned int polls = 0;
  while (true) {
    const long long idx = base - lane;
    const unsigned long long r = idx >= 0 ? vr[idx] : kP;  // before the first brick: prefix 0
    const unsigned int flag = (unsigned int)(r >> 62);
    const unsigned int pm = __ballot_sync(0xFFFFFFFFu, flag == 2u);
    const unsigned int zm = __ballot_sync(0xFFFFFFFFu, flag == 0u);
    const int lp = pm ? __ffs(pm) - 1 : 31;
    const unsigned int need = lp == 31 ? 0xFFFFFFFFu : ((2u << lp) - 1u);
    if (zm & need) {
      // a wait that ran out here or in another brick ends this one too
      if (++polls > kLookbackPolls || *reinterpret_cast<volatile int*>(errw) != 0) {
        if (lane == 0) atomicCAS(errw, 0, PC_ERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
      continue;
    }
    unsigned long long v = lane <= lp ? (r & kV) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    excl += v;
    if (pm) break;
    base -= 32;
  }
  if (lane == 0) vr[k] = kP | (excl + agg);
  return excl;
}

// Shared memory of k_compress (16-byte aligned regions): tables, codes with
// bound flags, padded centred inputs, Lorenzo codes (in the fixed-point form
// this region first holds the tensor-core A tiles of the two warpgroups),
// perceptron codes, histogram window, and the staged fixed-point network.
template <int BV, int MODE, int PV, int K, int H1, int H2>
struct CompLayout {
  static constexpr int G = BrickShape<BV>::G;
  static constexpr size_t a16(size_t v) { return (v + 15) & ~(size_t)15; }
  static constexpr size_t DQ = sizeof(Tabs);
  static constexpr size_t VP = DQ + a16((size_t)G * BV * 4);
  static constexpr size_t CZ = VP + a16((size_t)((G * PV + 3) & ~3) * 4);
  static constexpr size_t ATILES = MODE == 2 ? (size_t)2 * 2 * 128 * H1 * 2 : 0;  // 2 warpgroups x 2 limbs
  static constexpr size_t CN = CZ + a16((size_t)G * BV * 2 > ATILES ? (size_t)G * BV * 2 : ATILES);
  static constexpr size_t HI = CN + (MODE ? a16((size_t)G * BV * 2) : 0);
  static constexpr size_t ST = HI + (size_t)kHistWin * 4;
  static constexpr size_t TOTAL = ST + (MODE == 2 ? a16(sizeof(TcStage<H1 == 32 ? 32 : 16>)) : 0);
};

template <typename T, int B0, int B1, int B2, int MODE, int K, int H1, int H2>
__global__ void __launch_bounds__(256, MODE ? 2 : 3) k_compress(const __grid_constant__ CJobs jobs,
                                                                const __grid_constant__ Mlp mlp) {
  constexpr int BV = B0 * B1 * B2;
  using BS = BrickShape<BV>;
  constexpr int G = BS::G, TS = BS::TS, PPT = BS::PPT;
  constexpr bool WIDE = MODE != 0 && (K == 13 || K == 0);
  using PD = Pad<B0, B1, B2, WIDE>;
  constexpr int VW = (16 / (int)sizeof(T));
  constexpr bool VEC_OK = (B2 * G) % VW == 0;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int QK = MODE == 2 ? K : 7, QH = MODE == 2 ? H1 : 16;
  using CL = CompLayout<BV, MODE, PD::PV, K, H1, H2>;
  Tabs& tb = *reinterpret_cast<Tabs*>(smem);
  int* s_dq = reinterpret_cast<int*>(smem + CL::DQ);                   // G*BV: 2 q + ok
  int* s_vp = reinterpret_cast<int*>(smem + CL::VP);                   // G*PV padded inputs
  uint16_t* s_cz = reinterpret_cast<uint16_t*>(smem + CL::CZ);         // G*BV (after the A tiles)
  uint16_t* s_cn = reinterpret_cast<uint16_t*>(smem + CL::CN);         // G*BV (perceptron only)
  unsigned int* s_hist = reinterpret_cast<unsigned int*>(smem + CL::HI);
  // fixed-point form: staged network, tensor-core A tiles (over the Lorenzo codes)
  TcStage<QH>& tcs = *reinterpret_cast<TcStage<QH>*>(smem + CL::ST);
  uint8_t* s_atile = smem + CL::CZ;
  __shared__ int s_cost[G][2];
  __shared__ int s_nz[G];
  __shared__ unsigned int s_hz;  // the histogram's symbol 0 (balance points), from the per-block counts
  __shared__ int s_da[G];
  __shared__ int s_e2b[G];  // extent along x of each block of the brick (0: beyond the field)

  const int tid = threadIdx.x;
  for (int i = tid; i < G * PD::PV; i += 256) s_vp[i] = 0;
  for (int i = tid; i < kHistWin; i += 256) s_hist[i] = 0u;
  if (tid == 0) s_hz = 0u;
  const float sig = MODE ? __uint_as_float((unsigned int)(127 - mlp.s_in) << 23) : 1.0f;
  const float unsig = MODE ? __uint_as_float((unsigned int)(127 + mlp.s_in) << 23) : 1.0f;
  // fixed-point form: TMEM for the two warpgroups' accumulators (2 limbs x QH
  // columns each); the network is staged per field
  constexpr uint32_t kTmemCols = QH == 32 ? 128 : 64;
  uint32_t tmem_base = 0, tc_phase = 0;
  bool tc_ok = true;
  if constexpr (MODE == 2) {
    if (tid < 32) {
      tc::tmem_alloc(&tcs.tmem, kTmemCols);
      tc::tmem_relinquish();
    }
    if (tid == 0) {
      tc::mbar_init(&tcs.mbar[0], 1);
      tc::mbar_init(&tcs.mbar[1], 1);
      tc::mbar_init_fence();
    }
    tc::fence_before_sync();
  }
  __syncthreads();
  if constexpr (MODE == 2) {
    tc::fence_after_sync();
    tmem_base = tcs.tmem;
  }
  __shared__ int s_skip;
  // the current field (in shared memory, reloaded uniformly over the CTA when
  // the brick sequence enters the next field; kept out of registers)
  __shared__ CJob s_job;
  int jcur = -1;
  const Geo& g = s_job.g;
  uint16_t* const& codes = s_job.codes;
  uint8_t* const& nnflag = s_job.nnflag;
  uint32_t* const& nout = s_job.nout;
  unsigned long long* const& hist = s_job.hist;
  int* errw = nullptr;
  State c;
  int R = 2;
  bool jskip = true;
  // per-field scalars of the brick loop, also in shared memory
  __shared__ long long s_nbx, s_jb0;
  __shared__ int s_m, s_vec;
  const long long& nbx = s_nbx;
  const int& m = s_m;
  int hbase = 0;
  auto flush_hist = [&]() {
    __syncthreads();
    for (int i = tid; i < kHistWin; i += 256) {
      const unsigned int h = s_hist[i];
      if (h && hbase + i < (1 << m)) atomicAdd(&hist[hbase + i], (unsigned long long)h);
      s_hist[i] = 0u;
    }
    if (tid == 0) {
      if (s_hz) atomicAdd(&hist[0], (unsigned long long)s_hz);
      s_hz = 0u;
    }
  };
  const int team = tid / TS, t = tid % TS;
  int* dq = s_dq + team * BV;
  int* vp = s_vp + team * PD::PV;
  // single pass: bricks in order from the launch's counter; per-block bit and
  // balance counts, look-back results and team-scan scratch
  const bool sp = jobs.next != nullptr;
  __shared__ long long s_gbk;
  __shared__ unsigned int s_bbits[G], s_bout[G], s_scr[16];
  __shared__ unsigned long long s_pre[2];
  auto next_brick = [&](long long cur) -> long long {
    if (!sp) return cur + gridDim.x;
    __syncthreads();  // every thread has read the previous index
    if (tid == 0) s_gbk = (long long)atomicAdd(jobs.next, 1ull);
    __syncthreads();
    return s_gbk;
  };
  const long long gbk_first = sp ? next_brick(-1) : (long long)blockIdx.x;
  for (long long gbk = gbk_first; gbk < jobs.total; gbk = next_brick(gbk)) {
    int jn = jcur < 0 ? 0 : jcur;
    while (jn + 1 < jobs.n && gbk >= jobs.j[jn + 1].brick0) ++jn;
    if (jn != jcur) {
      if (jcur >= 0 && !jskip) flush_hist();
      const CJob& J = jobs.j[jn];
      jcur = jn;
      __syncthreads();  // the previous field's last brick is done with the tables and s_job
      if (tid == 0) s_job = J;
      errw = const_cast<int*>(&J.st->err);
      R = 1 << (J.m - 1);
      hbase = R - kHistWin / 2 > 0 ? R - kHistWin / 2 : 0;
      if (tid == 0) {
        s_m = J.m;
        s_nbx = (J.g.nb[2] + G - 1) / G;
        s_jb0 = J.brick0;
        s_vec = VEC_OK && (J.g.n[2] % VW == 0) && ((reinterpret_cast<uintptr_t>(J.x) & 15u) == 0);
        s_skip = J.st->err != 0;
      }
      c.Kp = J.st->Kp; c.Kn = J.st->Kn; c.Zq = J.st->Zq; c.S = J.st->S;
      c.step32 = J.st->step32; c.inv32 = J.st->inv32; c.ebdn32 = J.st->ebdn32;
      c.stepd = J.st->stepd; c.invd = J.st->invd; c.ebdnd = J.st->ebdnd;
      for (int i = tid; i < (int)(sizeof(Tabs) / 4); i += 256)
        reinterpret_cast<float*>(&tb)[i] = reinterpret_cast<const float*>(J.tabs)[i];
      if constexpr (MODE == 2) tcnet_stage<QK, QH>(J.qnet, tcs);
      __syncthreads();
      jskip = s_skip != 0;
    }
    if (jskip) continue;
    const long long brick = gbk - s_jb0;
    const bool vec_rows = s_vec != 0;
    const long long bxg = brick % nbx;
    const long long byz = brick / nbx;
    const long long by = byz % g.nb[1];
    const long long bz = byz / g.nb[1];
    const long long z0 = bz * B0, y0 = by * B1, x0 = bxg * G * B2;
    const int e0 = (int)min((long long)B0, g.n[0] - z0);
    const int e1 = (int)min((long long)B1, g.n[1] - y0);
    const int W = (int)min((long long)(G * B2), g.n[2] - x0);
    // a4: load the brick into registers (16-byte loads where rows allow), the
    // G block anchors first; then transform every point and write its code
    // (2 q + ok) and its anchor-centred clamped input in the padded block.
    constexpr int EPT = (G * BV + 255) / 256;  // elements per thread, <= 16
    constexpr int RW = G * B2 / VW;               // 16-byte vectors per brick row
    constexpr int NV = B0 * B1 * RW;
    const bool fullb = e0 == B0 && e1 == B1 && W == G * B2;
    // whole-vector rows only when a thread's vectors fit its EPT registers
    // (small bricks of 512 points have 2 elements per thread, fewer than one vector)
    constexpr bool VEC_FITS = ((NV + 255) / 256) * VW <= EPT;
    const bool vecb = VEC_FITS && fullb && vec_rows;
    const long long n12 = g.n[1] * g.n[2];
    const T* base = static_cast<const T*>(s_job.x) + z0 * n12 + y0 * g.n[2] + x0;
    T vals[EPT];
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int i = 0; i < EPT; ++i) vals[i] = T(0);  // elements a thread does not load stay defined
    }
    if (vecb) {
#pragma unroll
      for (int it = 0; it < (NV + 255) / 256; ++it) {
        const int e = tid + 256 * it;
        if (e < NV) {
          const int r = e / RW, cv = e % RW;
          const uint4 u = __ldg(reinterpret_cast<const uint4*>(base + (r / B1) * n12 + (r % B1) * g.n[2]) + cv);
          memcpy(&vals[it * VW], &u, 16);
        }
      }
    } else {
      const int tot = e0 * e1 * W;
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const int e = tid + 256 * i;
        if (e < tot) {
          const int r = e / W, col = e - r * W;
          vals[i] = __ldg(&base[(r / e1) * n12 + (r % e1) * g.n[2] + col]);
        }
      }
      // truncated blocks: padded cells outside the block read 0
      for (int i = tid; i < G * BV; i += 256) {
        const int gb = i / BV, j = i % BV;
        const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
        const int e2b = (int)min((long long)B2, g.n[2] - (bxg * G + gb) * B2);
        if (!(lz < e0 && ly < e1 && lx < e2b)) s_vp[gb * PD::PV + PD::at(lz, ly, lx)] = 0;
      }
    }
    if (tid < G) {
      int qa = 0;
      const long long bxt = bxg * G + tid;
      if (bxt < g.nb[2]) {
        bool okk;
        qa = Num<T>::transform(__ldg(&base[tid * B2]), c, tb, okk);
      }
      s_da[tid] = qa;
      s_e2b[tid] = bxt < g.nb[2] ? (int)min((long long)B2, g.n[2] - bxt * B2) : 0;
      s_cost[tid][0] = 0; s_cost[tid][1] = 0; s_nz[tid] = 0;
    }
    __syncthreads();
    // float64: every element's transform first (branch-free, independent
    // chains on the narrow FP64 unit): codes and a mask of ok
    int qv[sizeof(T) == 8 ? EPT : 1];
    unsigned int okm = 0;
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        bool ok;
        qv[i] = Num<T>::transform(vals[i], c, tb, ok);
        okm |= (ok ? 1u : 0u) << i;
      }
    }
    auto emit = [&](int vi, int row, int col) {
      const int gb = col / B2, lx = col % B2;
      const int lz = row / B1, ly = row % B1;
      int q, dq;
      if constexpr (sizeof(T) == 8) {
        q = qv[vi];
        dq = 2 * q + (int)((okm >> vi) & 1u);
      } else {
        bool ok;
        q = Num<T>::transform(vals[vi], c, tb, ok);
        dq = 2 * q + (ok ? 1 : 0);
      }
      s_dq[gb * BV + row * B2 + lx] = dq;
      s_vp[gb * PD::PV + PD::at(lz, ly, lx)] = clampd(q, s_da[gb]);
    };
    if (vecb) {
#pragma unroll
      for (int it = 0; it < (NV + 255) / 256; ++it) {
        const int e = tid + 256 * it;
        if (e < NV) {
          const int r = e / RW, cv = e % RW;
#pragma unroll
          for (int q = 0; q < VW; ++q) emit(it * VW + q, r, cv * VW + q);
        }
      }
    } else {
      const int tot = e0 * e1 * W;
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const int e = tid + 256 * i;
        if (e < tot) {
          const int r = e / W, col = e - r * W;
          emit(i, (r / e1) * B1 + (r % e1), col);
        }
      }
    }
    __syncthreads();
    if constexpr (MODE == 2) {
      // a6-a8, fixed-point form: tiles of 128 points on the tensor cores, one
      // per warpgroup at a time; each point's perceptron code and cost
      const int wg = tid >> 7, r = tid & 127;
      uint8_t* abuf = s_atile + (size_t)wg * 2 * 128 * QH * 2;
      const uint32_t tm = tmem_base + (uint32_t)(wg * 2 * QH);
      for (int tile = wg; tile < G * BV / 128; tile += 2) {
        const int f = tile * 128 + r;
        const int gb = f / BV, j = f - gb * BV;
        const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
        const int pj = gb * PD::PV + PD::at(lz, ly, lx);
        int xin[QK];
#pragma unroll
        for (int q = 0; q < QK; ++q) xin[q] = s_vp[pj + PD::off(st_dz(QK, q), st_dy(QK, q), st_dx(QK, q))];
        int prd;
        tc_ok &= tcnet_tile<QK, QH>(tcs, abuf, tm, wg, r, tc_phase, xin, tcs.mul512, prd);
        const bool valid = j != 0 && lz < e0 && ly < e1 && lx < s_e2b[gb];
        uint16_t coden = 0;
        int costn = 0;
        if (valid) {
          const int pd = s_dq[f];
          const int v = (pd >> 1) - s_da[gb];
          const int vk = v > (1 << 30) ? (1 << 30) : (v < -(1 << 30) ? -(1 << 30) : v);
          const long long kn = (long long)vk - (long long)prd;
          const long long an = kn < 0 ? -kn : kn;
          costn = bitlen_u((unsigned int)(an < R ? an : R));
          coden = (an <= R - 1 && (pd & 1)) ? (uint16_t)(kn + R) : 0;
        }
        s_cn[f] = coden;
        // the 32 points of a warp lie in one block
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) costn += __shfl_xor_sync(0xFFFFFFFFu, costn, o);
        if ((tid & 31) == 0 && costn) atomicAdd(&s_cost[gb][1], costn);
      }
      __syncthreads();
      if (!tc_ok) {
        atomicExch(errw, PC_ERR_TIMEOUT);
        tc_ok = true;
      }
    }
    const long long bx = bxg * G + team;
    const bool bvalid = bx < g.nb[2];
    const int e2 = bvalid ? (int)min((long long)B2, g.n[2] - bx * B2) : 0;
    const bool bfull = e0 == B0 && e1 == B1 && e2 == B2;
    const int da = s_da[team];
    // a6-a8: predict, quantize, cost (and, for Lorenzo only, a9 histogram)
    const long long b = (bz * g.nb[1] + by) * g.nb[2] + bx;
    int cz = 0, cn = 0, nz = 0;
    if constexpr (MODE == 1 && K > 0) {
      // two points per step through the packed perceptron forward
      if (bvalid) {
#pragma unroll 1
        for (int i = 0; i < PPT; i += 2) {
          int inp[2][K];
          int vks[2], js[2];
          bool oks[2], vals[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int j = t + (i + u) * TS;
            const bool inr = i + u < PPT && j < BV;
            js[u] = inr ? j : -1;
            const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
            const bool valid = inr && (bfull || (lz < e0 && ly < e1 && lx < e2)) && j != 0;
            vals[u] = valid;
            uint16_t codez = 0;
            int vk = 0;
            bool okp = false;
            if (valid) {
              const int pd = dq[j];
              okp = pd & 1;
              const int v = (pd >> 1) - da;
              vk = v > (1 << 30) ? (1 << 30) : (v < -(1 << 30) ? -(1 << 30) : v);
              const int pj = PD::at(lz, ly, lx);
              int lzp = 0;
#pragma unroll
              for (int q = 0; q < 7; ++q) lzp += lz_w(7, q) * vp[pj + PD::off(s7_dz(q), s7_dy(q), s7_dx(q))];
              const int kz = vk - lzp;
              const int az = kz < 0 ? -kz : kz;
              cz += bitlen_u((unsigned int)(az < R ? az : R));
              codez = (az <= R - 1 && okp) ? (uint16_t)(kz + R) : 0;
#pragma unroll
              for (int q = 0; q < K; ++q) inp[u][q] = vp[pj + PD::off(st_dz(K, q), st_dy(K, q), st_dx(K, q))];
            } else {
#pragma unroll
              for (int q = 0; q < K; ++q) inp[u][q] = 0;
            }
            vks[u] = vk;
            oks[u] = okp;
            if (inr) s_cz[team * BV + j] = codez;
          }
          float pv[2];
          mlp_fwd2<K, H1, H2>(mlp, inp[0], inp[1], sig, unsig, pv[0], pv[1]);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            uint16_t coden = 0;
            if (vals[u]) {
              const long long kn = (long long)vks[u] - (long long)round_pred(pv[u]);
              const long long an = kn < 0 ? -kn : kn;
              cn += bitlen_u((unsigned int)(an < R ? an : R));
              coden = (an <= R - 1 && oks[u]) ? (uint16_t)(kn + R) : 0;
            }
            if (js[u] >= 0) s_cn[team * BV + js[u]] = coden;
          }
        }
      }
    } else if (bvalid) {
#pragma unroll(MODE ? 1 : PPT)
      for (int i = 0; i < PPT; ++i) {
        const int j = t + i * TS;
        if (j >= BV) break;
        const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
        const bool valid = (bfull || (lz < e0 && ly < e1 && lx < e2)) && j != 0;
        uint16_t codez = 0, coden = 0;
        if (valid) {
          const int pd = dq[j];
          const bool okp = pd & 1;
          const int v = (pd >> 1) - da;                          // |v| < 2^31
          const int vk = v > (1 << 30) ? (1 << 30) : (v < -(1 << 30) ? -(1 << 30) : v);
          const int pj = PD::at(lz, ly, lx);
          int lzp = 0;
#pragma unroll
          for (int q = 0; q < 7; ++q) lzp += lz_w(7, q) * vp[pj + PD::off(s7_dz(q), s7_dy(q), s7_dx(q))];
          const int kz = vk - lzp;
          const int az = kz < 0 ? -kz : kz;
          cz += bitlen_u((unsigned int)(az < R ? az : R));
          codez = (az <= R - 1 && okp) ? (uint16_t)(kz + R) : 0;
          if constexpr (MODE == 1) {
            long long prd;
            {
              constexpr int KK = K > 0 ? K : 13;
              int in[KK];
              const int kk = K > 0 ? K : mlp.k;
#pragma unroll
              for (int q = 0; q < KK; ++q)
                in[q] = q < kk ? vp[pj + PD::off(st_dz(kk, q), st_dy(kk, q), st_dx(kk, q))] : 0;
              float pv;
              if constexpr (K > 0) pv = mlp_fwd<K, H1, H2>(mlp, in, sig, unsig);
              else pv = mlp_fwd_rt(mlp, in, sig, unsig);
              prd = round_pred(pv);
            }
            const long long kn = (long long)vk - prd;
            const long long an = kn < 0 ? -kn : kn;
            cn += bitlen_u((unsigned int)(an < R ? an : R));
            coden = (an <= R - 1 && okp) ? (uint16_t)(kn + R) : 0;
          } else if constexpr (MODE == 0) {
            if (!sp) {
              nz += codez == 0;
              // balance points (code 0, most points of a field the predictors miss) are
              // counted per block, not one atomic each on a single bin
              const int hi = (int)codez - hbase;
              if (codez != 0) {
                if (hi >= 0 && hi < kHistWin) atomicAdd(&s_hist[hi], 1u);
                else atomicAdd(&hist[codez], 1ull);
              }
            }
          }
        }
        s_cz[team * BV + j] = codez;
        if constexpr (MODE == 1) s_cn[team * BV + j] = coden;
      }
    }
    // team sums (the fixed-point form summed its perceptron costs per warp)
    int tcz = team_sum<TS>(cz, &s_cost[team][0]);
    int tcn = MODE == 1 ? team_sum<TS>(cn, &s_cost[team][1]) : 0;
    int tnz = MODE ? 0 : team_sum<TS>(nz, &s_nz[team]);
    __syncthreads();
    if constexpr (TS != 32) {
      tcz = s_cost[team][0];
      tcn = s_cost[team][1];
      tnz = s_nz[team];
    }
    if constexpr (MODE == 2) tcn = s_cost[team][1];
    if (sp) {
      // a7 select and a8-a12 in one pass: codes outside the codebook become
      // balance points; each block's bits and balance points are counted,
      // the brick's stream and balance offsets come from a look-back over
      // the bricks before it, and the brick's code words are packed on chip
      // and written with its block-table entries and balance values.
      const bool usen = MODE != 0 && tcn < tcz;
      uint16_t* srcw = (usen ? s_cn : s_cz) + team * BV;
      constexpr int CPT = BV / TS;
      const uint32_t* cwl = s_job.cwl;
      const unsigned int cw0 = __ldg(cwl);  // symbol 0: always in the codebook
      unsigned int nbits = 0, nzero = 0;
      if (bvalid) {
#pragma unroll 4
        for (int i = 0; i < CPT; ++i) {
          const int j = t * CPT + i;
          const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
          const bool valid = (bfull || (lz < e0 && ly < e1 && lx < e2)) && j != 0;
          if (valid) {
            unsigned int cd = srcw[j];
            unsigned int e = __ldg(cwl + cd);
            if ((e >> 24) == 0u) {
              cd = 0u;
              e = cw0;
              srcw[j] = 0;
            }
            nbits += e >> 24;
            nzero += cd == 0u;
          }
        }
      }
      unsigned int pb, po, tbits, tzero;
      team_exscan2<TS>(nbits, nzero, pb, po, tbits, tzero, s_scr);
      if (t == 0) {
        s_bbits[team] = bvalid ? tbits : 0u;
        s_bout[team] = bvalid ? 1u + tzero : 0u;
      }
      __syncthreads();
      if (bvalid && t == 0) {
        st_u32(s_job.out + s_job.off_bb + 4ull * b, tbits | (usen ? 0x80000000u : 0u));
        *reinterpret_cast<uint16_t*>(s_job.out + s_job.off_bn + 2ull * b) = (uint16_t)(1u + tzero);
      }
      if (tid < 64) {
        // warp 0: stream bits, warp 1: balance points
        const int w = tid >> 5, lane = tid & 31;
        unsigned long long agg = 0;
#pragma unroll
        for (int q = 0; q < G; ++q) agg += w ? s_bout[q] : s_bbits[q];
        const unsigned long long ex = lookback(s_job.rec + (w ? s_job.nbk : 0), brick, agg, lane, errw);
        if (lane == 0) s_pre[w] = ex;
      }
      __syncthreads();
      const unsigned long long S = s_pre[0], O = s_pre[1];
      unsigned int bo = 0, oo = 0, btot = 0;
#pragma unroll
      for (int q = 0; q < G; ++q) {
        if (q < team) { bo += s_bbits[q]; oo += s_bout[q]; }
        btot += s_bbits[q];
      }
      const unsigned int sh = (unsigned int)(S & 31ull);
      const int nwords = (int)((sh + btot + 31u) >> 5);
      unsigned int* buf = reinterpret_cast<unsigned int*>(s_dq);  // the brick's words (codes are done)
      for (int i = tid; i < nwords; i += 256) buf[i] = 0u;
      __syncthreads();
      if (bvalid) {
        T* ov = static_cast<T*>(s_job.ov);
        const T* org = base + team * B2;  // the block's first point
        unsigned long long o = O + oo;
        if (t == 0) ov[o] = org[0];       // the anchor, first of the block's balance values
        o += 1ull + po;
        unsigned int p = sh + bo + pb;
#pragma unroll 4
        for (int i = 0; i < CPT; ++i) {
          const int j = t * CPT + i;
          const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
          const bool valid = (bfull || (lz < e0 && ly < e1 && lx < e2)) && j != 0;
          if (valid) {
            const unsigned int cd = srcw[j];
            const unsigned int e = __ldg(cwl + cd);
            const unsigned int L = e >> 24, wv = e & 0xFFFFFFu;
            const unsigned int wi = p >> 5, bb2 = p & 31u;
            if (bb2 + L <= 32u) {
              atomicOr(&buf[wi], wv << (32u - bb2 - L));
            } else {
              atomicOr(&buf[wi], wv >> (bb2 + L - 32u));
              atomicOr(&buf[wi + 1], wv << (64u - bb2 - L));
            }
            p += L;
            if (cd == 0u) ov[o++] = org[lz * n12 + ly * g.n[2] + lx];
          }
        }
      }
      __syncthreads();
      if (btot) {
        // whole words go straight out; a word shared with a neighbouring
        // brick is kept aside and assembled once every brick is done
        uint32_t* stream = reinterpret_cast<uint32_t*>(s_job.out + s_job.off_st);
        const unsigned long long W0 = S >> 5;
        const bool head_part = sh != 0u, tail_part = ((sh + btot) & 31u) != 0u;
        if (W0 + (unsigned long long)nwords > s_job.cap_words) {
          if (tid == 0) atomicExch(errw, PC_ERR_CAPACITY);
        } else {
          for (int i = tid; i < nwords; i += 256) {
            const bool part = (i == 0 && head_part) || (i == nwords - 1 && tail_part);
            if (!part) stream[W0 + i] = buf[i];
          }
        }
        if (tid == 0) {
          s_job.side[2 * brick] = buf[0];
          s_job.side[2 * brick + 1] = buf[nwords - 1];
        }
      }
      __syncthreads();
      continue;
    }
    // a7 select, a8 emit, a9 histogram of the chosen codes
    if (bvalid) {
      const bool usen = MODE != 0 && tcn < tcz;
      const uint16_t* src = usen ? s_cn + team * BV : s_cz + team * BV;
      if constexpr (MODE != 0) {
        int nzz = 0;
#pragma unroll 4
        for (int i = 0; i < PPT; ++i) {
          const int j = t + i * TS;
          if (j < BV) {
            const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
            const bool valid = (bfull || (lz < e0 && ly < e1 && lx < e2)) && j != 0;
            if (valid) {
              const uint16_t cd = src[j];
              nzz += cd == 0;
              const int hi = (int)cd - hbase;
              if (cd != 0) {  // code 0: counted per block
                if (hi >= 0 && hi < kHistWin) atomicAdd(&s_hist[hi], 1u);
                else atomicAdd(&hist[cd], 1ull);
              }
            }
          }
        }
        tnz = team_sum<TS>(nzz, &s_nz[team]);
      }
      uint4* dst = reinterpret_cast<uint4*>(codes + b * BV);
      const uint4* sv = reinterpret_cast<const uint4*>(src);
      for (int i = t; i < BV / 8; i += TS) dst[i] = sv[i];
    }
    if constexpr (MODE != 0 && TS != 32) {
      __syncthreads();
      tnz = s_nz[team];
    }
    if (bvalid && t == 0) {
      nnflag[b] = (MODE != 0 && tcn < tcz) ? 1 : 0;
      nout[b] = 1u + (unsigned int)tnz;
      if (tnz) atomicAdd(&s_hz, (unsigned int)tnz);
    }
    __syncthreads();
  }
  if (jcur >= 0 && !jskip) flush_hist();
  if constexpr (MODE == 2) {
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem_base, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers (called from the API layer).
// ---------------------------------------------------------------------------
template <typename T>
int launch_stats_consts(const void* x, unsigned long long n, State* st, Tabs* tabs, unsigned long long* hist,
                        int nsym, double eb, int nsm, cudaStream_t s) {
  { ProfScope p(kStInit, s); k_init<<<64, 256, 0, s>>>(st, hist, nsym); }
  { ProfScope p(kStStats, s); k_stats<T><<<nsm * 8, 256, 0, s>>>(static_cast<const T*>(x), n, st); }
  { ProfScope p(kStConsts, s); k_consts<T><<<1, 128, 0, s>>>(st, eb, tabs); }
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
template int launch_stats_consts<float>(const void*, unsigned long long, State*, Tabs*, unsigned long long*, int,
                                        double, int, cudaStream_t);
template int launch_stats_consts<double>(const void*, unsigned long long, State*, Tabs*, unsigned long long*, int,
                                         double, int, cudaStream_t);

template <typename T, int B0, int B1, int B2, int MODE, int K, int H1, int H2>
static int launch_c(const CJobs& jobs, const Mlp& mlp, int nsm, cudaStream_t s) {
  constexpr int BV = B0 * B1 * B2;
  constexpr bool WIDE = MODE != 0 && (K == 13 || K == 0);
  auto kern = k_compress<T, B0, B1, B2, MODE, K, H1, H2>;
  constexpr size_t sm = CompLayout<BV, MODE, Pad<B0, B1, B2, WIDE>::PV, K, H1, H2>::TOTAL;
  static_assert(sm <= 232448, "shared memory per CTA");
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return PC_ERR_CUDA;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
  if constexpr (MODE == 2) {
    // the whole unified L1 as shared memory, so that two CTAs fit on an SM
    if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
      return PC_ERR_CUDA;
    // The occupancy query reports one CTA per SM for the tensor-core form;
    // registers (launch bounds) and shared memory allow two, and two CTAs
    // hold 2 x 128 (or 2 x 64) of the 512 TMEM columns.
    const int by_smem = (int)((228u << 10) / (sm + 2048));
    per_sm = by_smem >= 2 ? 2 : 1;
  }
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)nsm * per_sm;
  if (grid > jobs.total) grid = jobs.total;
  if (grid < 1) grid = 1;
  {
    ProfScope p(kStCompress, s);
    kern<<<(unsigned int)grid, 256, sm, s>>>(jobs, mlp);
  }
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

template <typename T, int B0, int B1, int B2>
static int launch_c_shape(const CJobs& jobs, int mode, const Mlp& mlp, int nsm, cudaStream_t s) {
  if (mode == 0) return launch_c<T, B0, B1, B2, 0, 0, 0, 0>(jobs, mlp, nsm, s);
  if (mode == 2) {
    if (mlp.k == 7 && mlp.h1 == 16 && mlp.h2 == 16) return launch_c<T, B0, B1, B2, 2, 7, 16, 16>(jobs, mlp, nsm, s);
    if (mlp.k == 13 && mlp.h1 == 32 && mlp.h2 == 32) return launch_c<T, B0, B1, B2, 2, 13, 32, 32>(jobs, mlp, nsm, s);
    return PC_ERR_ARG;
  }
  if (mlp.k == 7 && mlp.h1 == 16 && mlp.h2 == 16) return launch_c<T, B0, B1, B2, 1, 7, 16, 16>(jobs, mlp, nsm, s);
  if (mlp.k == 13 && mlp.h1 == 32 && mlp.h2 == 32) return launch_c<T, B0, B1, B2, 1, 13, 32, 32>(jobs, mlp, nsm, s);
  return launch_c<T, B0, B1, B2, 1, 0, 0, 0>(jobs, mlp, nsm, s);
}

template <typename T>
int launch_compress(const CJob* jl, int n, int mode, const Mlp& mlp, int nsm, cudaStream_t s,
                    unsigned long long* next) {
  if (n < 1 || n > kMaxJobs) return PC_ERR_ARG;
  static thread_local CJobs jobs;
  jobs.n = n;
  jobs.total = 0;
  jobs.next = next;
  const Geo& g = jl[0].g;
  for (int i = 0; i < n; ++i) {
    if (jl[i].g.b[0] != g.b[0] || jl[i].g.b[1] != g.b[1] || jl[i].g.b[2] != g.b[2]) return PC_ERR_ARG;
    jobs.j[i] = jl[i];
    jobs.j[i].brick0 = jobs.total;
    jobs.total += bricks_of(jl[i].g);
  }
  const int b0 = g.b[0], b1 = g.b[1], b2 = g.b[2];
#define PC_SHAPE(A, B, C) \
  if (b0 == A && b1 == B && b2 == C) return launch_c_shape<T, A, B, C>(jobs, mode, mlp, nsm, s);
  PC_SHAPE(8, 8, 8)
  PC_SHAPE(4, 4, 4)
  PC_SHAPE(16, 16, 16)
  PC_SHAPE(1, 16, 32)
  PC_SHAPE(1, 8, 8)
  PC_SHAPE(1, 64, 64)
#undef PC_SHAPE
  return PC_ERR_ARG;
}
template int launch_compress<float>(const CJob*, int, int, const Mlp&, int, cudaStream_t, unsigned long long*);
template int launch_compress<double>(const CJob*, int, int, const Mlp&, int, cudaStream_t, unsigned long long*);

}  // namespace pc
