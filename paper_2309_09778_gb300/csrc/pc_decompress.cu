// a13: the inverse path (Section V, decompression).
//
// k_dec_tables rebuilds the canonical decoder from the stored (symbol, length)
// list and validates it; k_dec_chunksum / k_dec_chunkscan / k_dec_blockoff
// turn the block table into per-block bit and balance-point offsets;
// k_huff_decode decodes one block per thread (the same step for
// every code: a 12-bit length table, register compares for longer codes),
// checking every read against the block's stated bit count; k_recon rebuilds
// each block along wavefronts of its causal stencil with the same predictor
// and inverse map as the compressor, then writes the brick with coalesced
// stores.  A damaged stream sets the error word and never leads to an
// out-of-bounds access.
#include "pc_kernels.cuh"
#include "pc_qmlp.cuh"
#include "pc_tcnet.cuh"
#include "pc_profile.cuh"

namespace pc {

// The stored list is the code order (lengths never decrease along it), so the
// decoder tables follow from one pass: the symbol at list position p has code
// first[len] + (p - offset[len]).  Each length's count is the distance from its
// first position to the next length's; a position whose length differs from
// its predecessor's marks a first position (one writer per length).
__global__ void __launch_bounds__(1024) k_dec_tables(const uint8_t* __restrict__ in, DecInfo di, DecScratch ds) {
  __shared__ unsigned int s_start[32];
  __shared__ unsigned int s_seen[2048];  // one bit per symbol (m <= 16)
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nsym = 1 << di.m;
  const int n = (int)di.n_used;
  if (tid < 32) s_start[tid] = 0xFFFFFFFFu;
  if (tid == 0) s_bad = 0;
  if (tid < 128) build_tabs_entry(ds.ftab, tid);
  for (int i = tid; i < 2048; i += nt) s_seen[i] = 0u;
  __syncthreads();
  const unsigned int* ent = reinterpret_cast<const unsigned int*>(in + di.off_cb);
  // four entries per thread and step, their loads issued together
  constexpr int U = 4;
  for (int p0 = tid; p0 < n; p0 += U * nt) {
    unsigned int e[U], pe[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int p = p0 + k * nt;
      e[k] = p < n ? ent[p] : 0u;
      pe[k] = p > 0 && p < n ? ent[p - 1] : 0u;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int p = p0 + k * nt;
      if (p >= n) break;
      const unsigned int sym = e[k] & 0xFFFFu, len = e[k] >> 16, prev = pe[k] >> 16;
      bool bad = sym >= (unsigned int)nsym || len < 1 || len > (unsigned int)kLmax || len < prev;
      if (!bad) {
        const unsigned int bit = 1u << (sym & 31u);
        bad |= (atomicOr(&s_seen[sym >> 5], bit) & bit) != 0u;
      }
      if (bad) { s_bad = 1; continue; }
      ds.sorted[p] = (uint16_t)sym;
      if (len != prev) s_start[len] = (unsigned int)p;
    }
  }
  __syncthreads();
  if (s_bad) { if (tid == 0) atomicExch(ds.err, PC_ERR_CORRUPT); return; }
  if (tid == 0) {
    unsigned int cnt[kLmax + 1];
    unsigned int next = (unsigned int)n;
    for (int l = kLmax; l >= 1; --l) {
      const unsigned int st = s_start[l];
      cnt[l] = st != 0xFFFFFFFFu ? next - st : 0u;
      if (st != 0xFFFFFFFFu) next = st;
    }
    unsigned int code = 0, off = 0;
    bool bad = false;
    for (int l = 1; l <= kLmax; ++l) {
      const unsigned int prevc = l > 1 ? cnt[l - 1] : 0u;
      code = (code + prevc) << 1;
      off += prevc;
      ds.tabs[l] = code;        // first code of length l
      ds.tabs[32 + l] = cnt[l];  // count
      ds.tabs[64 + l] = off;     // list position of the first code of length l
      if (cnt[l] && (unsigned long long)code + cnt[l] > (1ull << l)) bad = true;
    }
    if (bad) atomicExch(ds.err, PC_ERR_CORRUPT);
  }
}

__device__ __forceinline__ void dec_block_coords(const Geo& g, long long b, long long& bz, long long& by,
                                                 long long& bx, int& e0, int& e1, int& e2) {
  bx = b % g.nb[2];
  const long long t = b / g.nb[2];
  by = t % g.nb[1];
  bz = t / g.nb[1];
  e0 = (int)min((long long)g.b[0], g.n[0] - bz * g.b[0]);
  e1 = (int)min((long long)g.b[1], g.n[1] - by * g.b[1]);
  e2 = (int)min((long long)g.b[2], g.n[2] - bx * g.b[2]);
}

__global__ void __launch_bounds__(256) k_dec_chunksum(Geo g, const uint8_t* __restrict__ in, DecInfo di,
                                                      DecScratch ds) {
  __shared__ unsigned long long s_b[8], s_o[8];
  const long long c = blockIdx.x;
  const long long b0 = c * g.ch, b1 = min(g.nblocks, b0 + g.ch);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long wb = 0, wo = 0;
  bool bad = false;
  for (long long b = b0 + threadIdx.x; b < b1; b += 256) {
    long long bz, by, bx;
    int e0, e1, e2;
    dec_block_coords(g, b, bz, by, bx, e0, e1, e2);
    const unsigned int npts = (unsigned int)(e0 * e1 * e2);
    const unsigned int bits = *reinterpret_cast<const unsigned int*>(in + di.off_bb + 4ull * b) & 0x7FFFFFFFu;
    const unsigned int no = *reinterpret_cast<const uint16_t*>(in + di.off_bn + 2ull * b);
    if (no < 1 || no > npts || bits > (npts - 1) * (unsigned int)kLmax) bad = true;
    wb += bits;
    wo += no;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wb += __shfl_xor_sync(0xFFFFFFFFu, wb, o);
    wo += __shfl_xor_sync(0xFFFFFFFFu, wo, o);
  }
  if (bad) atomicExch(ds.err, PC_ERR_CORRUPT);
  if (lane == 0) { s_b[wid] = wb; s_o[wid] = wo; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tb = 0, to = 0;
    for (int i = 0; i < 8; ++i) { tb += s_b[i]; to += s_o[i]; }
    ds.chunk_bits[c] = tb;
    ds.chunk_nout[c] = to;
  }
}

__global__ void __launch_bounds__(1024) k_dec_chunkscan(Geo g, DecInfo di, DecScratch ds) {
  __shared__ unsigned long long s_w[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long nc = g.nchunks;
  const long long per = (nc + nt - 1) / nt;
  const long long lo = min(nc, tid * per), hi = min(nc, lo + per);
  unsigned long long sb = 0, so = 0;
  for (long long i = lo; i < hi; ++i) { sb += ds.chunk_bits[i]; so += ds.chunk_nout[i]; }
  unsigned long long tb, to;
  unsigned long long pb = cta_exscan<unsigned long long>(sb, s_w, tb);
  unsigned long long po = cta_exscan<unsigned long long>(so, s_w, to);
  for (long long i = lo; i < hi; ++i) {
    ds.chunk_boff[i] = pb;
    ds.chunk_ooff[i] = po;
    pb += ds.chunk_bits[i];
    po += ds.chunk_nout[i];
  }
  if (tid == 0 && ((tb + 31) / 32 != di.swords || to != di.n_out)) atomicExch(ds.err, PC_ERR_CORRUPT);
}

__global__ void __launch_bounds__(256) k_dec_blockoff(Geo g, const uint8_t* __restrict__ in, DecInfo di,
                                                      DecScratch ds) {
  __shared__ unsigned int s_w[32];
  const long long c = blockIdx.x;
  const long long b0 = c * g.ch, b1 = min(g.nblocks, b0 + g.ch);
  const int nb = (int)(b1 - b0);
  const int tid = threadIdx.x;
  const int per = (nb + 255) / 256;
  const int lo = min(nb, tid * per), hi = min(nb, lo + per);
  unsigned int sb = 0, so = 0;
  for (int i = lo; i < hi; ++i) {
    sb += *reinterpret_cast<const unsigned int*>(in + di.off_bb + 4ull * (b0 + i)) & 0x7FFFFFFFu;
    so += *reinterpret_cast<const uint16_t*>(in + di.off_bn + 2ull * (b0 + i));
  }
  unsigned int tb, to;
  unsigned int pb = cta_exscan<unsigned int>(sb, s_w, tb);
  unsigned int po = cta_exscan<unsigned int>(so, s_w, to);
  const unsigned long long cb = ds.chunk_boff[c], co = ds.chunk_ooff[c];
  for (int i = lo; i < hi; ++i) {
    ds.boff[b0 + i] = cb + pb;
    ds.ooff[b0 + i] = co + po;
    pb += *reinterpret_cast<const unsigned int*>(in + di.off_bb + 4ull * (b0 + i)) & 0x7FFFFFFFu;
    po += *reinterpret_cast<const uint16_t*>(in + di.off_bn + 2ull * (b0 + i));
  }
}

// One thread per block: canonical Huffman decode into block-strided codes.
// The output is each code's position in the stored codebook list (the code
// order: lengths never decrease along it); the reconstruction maps positions
// to symbols when it stages a block.  Eight positions are packed and written with one 16-byte
// store.
constexpr int kDecThreads = 128;  // threads (blocks decoded) per CTA of k_huff_decode
constexpr int kShortBits = 12;    // codes up to this long take their length from a table

// The decoder of CTA `cta` of one field (kDecThreads blocks, one per thread).
__device__ __forceinline__ void huff_decode_cta(const Geo& g, const uint8_t* __restrict__ in, const DecInfo& di,
                                                const DecScratch& ds, long long cta) {
  // per length l: left-justified end of its code range (the ranges tile the
  // 24-bit window space in length order) and list position minus first code
  __shared__ unsigned int s_lim[32];
  __shared__ unsigned int s_base[32];
  // length of the code a 12-bit window prefix starts, 0 for longer codes
  __shared__ uint8_t s_len[1 << kShortBits];
  // per-lane stream window: 36 words from a 16-byte aligned word base, word-major
  // (the lanes of a warp read distinct banks whatever words they need)
  __shared__ unsigned int s_win[36][kDecThreads];
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    const int L = l + 1;
    s_lim[l] = L <= kLmax ? (ds.tabs[L] + ds.tabs[32 + L]) << (kLmax - L) : 0xFFFFFFFFu;
    s_base[l] = ds.tabs[64 + l] - ds.tabs[l];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (1 << kShortBits); i += blockDim.x) {
    // the shortest length whose range end is past every window with this prefix
    const unsigned int top = ((unsigned int)(i + 1) << (kLmax - kShortBits)) - 1u;
    int l = 1;
    while (l <= kShortBits && s_lim[l - 1] <= top) ++l;
    s_len[i] = (uint8_t)(l <= kShortBits ? l : 0);
  }
  __syncthreads();
  if (*ds.err) return;
  const long long b = cta * blockDim.x + threadIdx.x;
  if (b >= g.nblocks) return;
  // range ends of the long lengths, in registers
  unsigned int lim[kLmax - kShortBits];
#pragma unroll
  for (int k = 0; k < kLmax - kShortBits; ++k) lim[k] = s_lim[kShortBits + k];
  const unsigned int lim_short = s_lim[kShortBits - 1];  // windows below it start a short code
  long long bz, by, bx;
  int e0, e1, e2;
  dec_block_coords(g, b, bz, by, bx, e0, e1, e2);
  const bool full = e0 == g.b[0] && e1 == g.b[1] && e2 == g.b[2];
  const unsigned int nbits = *reinterpret_cast<const unsigned int*>(in + di.off_bb + 4ull * b) & 0x7FFFFFFFu;
  // Every 32 codes each lane copies the next 144 bytes of its stream (at
  // least 32 codes of at most 24 bits) into its shared-memory window with
  // independent 16-byte loads.  The stream section starts 16-byte aligned and
  // chunks past it read as zero.  Between refills the bits stream through a
  // 64-bit register buffer (hi:lo, next bit at bit 31 of hi) whose next word
  // is read one code ahead.
  const uint4* s4 = reinterpret_cast<const uint4*>(di.stream);
  const unsigned long long nq = (di.swords + 3) / 4;
  const unsigned int tid = threadIdx.x;
  const unsigned long long p0 = ds.boff[b];
  unsigned int hi = 0, lo = 0;
  int nb = 0;                      // valid bits in hi:lo, > 32 before each step
  unsigned int wi = 0, wnext = 0;  // next window word and its value
  unsigned int used = 0;           // bits consumed so far
  auto refill = [&]() {
    const unsigned long long p = p0 + used;
    const unsigned long long q0 = p >> 7;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const uint4 v = q0 + k < nq ? __ldg(s4 + q0 + k) : make_uint4(0u, 0u, 0u, 0u);
      s_win[4 * k][tid] = v.x;
      s_win[4 * k + 1][tid] = v.y;
      s_win[4 * k + 2][tid] = v.z;
      s_win[4 * k + 3][tid] = v.w;
    }
    const unsigned int w0 = (unsigned int)(p >> 5) & 3u;
    const unsigned int sh = (unsigned int)(p & 31ull);
    const unsigned int a0 = s_win[w0][tid], a1 = s_win[w0 + 1][tid], a2 = s_win[w0 + 2][tid];
    hi = __funnelshift_l(a1, a0, sh);
    lo = __funnelshift_l(a2, a1, sh);
    nb = 64 - (int)sh;
    wi = w0 + 2;
    wnext = a2;
  };
  bool bad = false;
  const unsigned int nused = di.n_used;
  // one decode step, the same for every code: short lengths from the table,
  // long ones by comparing the window with the long range ends
  auto step = [&]() -> unsigned int {
    const unsigned int peek = hi >> (32 - kLmax);
    int ll = kShortBits + 1;
#pragma unroll
    for (int k = 0; k < kLmax - kShortBits; ++k) ll += lim[k] <= peek ? 1 : 0;
    const int ls = s_len[peek >> (kLmax - kShortBits)];
    const int l = peek < lim_short ? ls : ll;
    bad |= l > kLmax;  // past the last code range: not a code
    const int lc = l <= kLmax ? l : kLmax;
    const unsigned int idx = s_base[lc] + (peek >> (kLmax - lc));
    hi = __funnelshift_l(lo, hi, (unsigned int)lc);
    lo <<= lc;
    nb -= lc;
    // below 33 valid bits, all of them are in hi: the next word goes right after
    const bool r = nb <= 32;
    const unsigned int s2 = (unsigned int)(32 - nb);
    hi |= r ? __funnelshift_l(wnext, 0u, s2) : 0u;
    lo |= r ? wnext << s2 : 0u;
    nb += r ? 32 : 0;
    wi += r ? 1u : 0u;
    wnext = s_win[wi < 35u ? wi : 35u][tid];
    used += (unsigned int)lc;
    return idx < nused ? idx : 0u;
  };
  uint4* out = reinterpret_cast<uint4*>(ds.codes + b * g.bvol);
  const int B1 = g.b[1], B2 = g.b[2];
  int lz0 = 0, ly0 = 0, lx0 = 0;  // block coordinates of slot j0
  for (int j0 = 0; j0 < g.bvol; j0 += 8) {
    if ((j0 & 31) == 0) refill();
    unsigned int sy[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      bool valid = j0 + q != 0;
      if (!full) {
        // slot j0 + q, one row wrap at most (rows hold at least 4 slots)
        int lx = lx0 + q, ly = ly0, lz = lz0;
        if (lx >= B2) {
          lx -= B2;
          if (++ly == B1) { ly = 0; ++lz; }
        }
        valid = valid && lz < e0 && ly < e1 && lx < e2;
      }
      sy[q] = (valid && !bad) ? step() : 0u;
    }
    unsigned int pk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) pk[q] = sy[2 * q] | (sy[2 * q + 1] << 16);
    out[j0 >> 3] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    lx0 += 8;
    while (lx0 >= B2) {
      lx0 -= B2;
      if (++ly0 == B1) { ly0 = 0; ++lz0; }
    }
  }
  // a corrupt stream shows as a window past every code range or a bit count
  // that differs from the block table's
  if (bad || used != nbits) atomicExch(ds.err, PC_ERR_CORRUPT);
}

__global__ void __launch_bounds__(kDecThreads) k_huff_decode(Geo g, const uint8_t* __restrict__ in, DecInfo di,
                                                     DecScratch ds) {
  huff_decode_cta(g, in, di, ds, blockIdx.x);
}

// Many fields in one launch: CTA c belongs to the last job whose first CTA is
// at most c (the job table travels as a kernel parameter).
__global__ void __launch_bounds__(kDecThreads) k_huff_decode_jobs(const __grid_constant__ DecJobs jobs) {
  int jn = 0;
  while (jn + 1 < jobs.n && (long long)blockIdx.x >= jobs.j[jn + 1].cta0) ++jn;
  const DecJob& J = jobs.j[jn];
  huff_decode_cta(J.g, J.in, J.di, J.ds, (long long)blockIdx.x - J.cta0);
}

int launch_huff_jobs(const DecJob* jl, int n, cudaStream_t s) {
  if (n < 1 || n > kMaxDecJobs) return PC_ERR_ARG;
  static thread_local DecJobs jobs;
  jobs.n = n;
  long long ctas = 0;
  for (int i = 0; i < n; ++i) {
    jobs.j[i] = jl[i];
    jobs.j[i].cta0 = ctas;
    ctas += (jl[i].g.nblocks + kDecThreads - 1) / kDecThreads;
  }
  if (ctas < 1) return PC_OK;
  ProfScope p(kStHuffDecode, s);
  k_huff_decode_jobs<<<(unsigned int)ctas, kDecThreads, 0, s>>>(jobs);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Wavefront reconstruction.  Schedule s(p) = z + y + x for the 7-point
// stencil and 4z + 2y + x for the 13-point one: every causal neighbour has a
// smaller s, so all points of one wave are independent.  Blocks are rebuilt in
// bricks (as in compression) in zero-bordered padded arrays, and the brick is
// written back with coalesced (16-byte where rows allow) stores.
// ---------------------------------------------------------------------------
// Blocks rebuilt together by one CTA.  The FP32 perceptron path flattens
// every wave over all of them, so its single-precision bricks of up to
// 512-point blocks take two groups of G (16 blocks, two CTAs per SM still
// fit): narrow waves are latency-bound, and more blocks per wave spread that
// latency over more points.
template <int BV, int TSZ, int MODE, int K>
constexpr int recon_blocks() {
  return BrickShape<BV>::G * ((MODE == 1 && K > 0 && BV <= 512 && TSZ == 4) ? 2 : 1);
}

// Shared-memory layout of k_recon (16-byte aligned regions).  The per-block
// strides are padded so that the same point of the GR blocks falls on
// different banks: wave positions run block-fastest across the lanes.
template <int B0, int B1, int B2, int PV, int TSZ, int MODE, int K, int H1, int H2>
struct ReconLayout {
  static constexpr int BV = B0 * B1 * B2;
  static constexpr int GR = recon_blocks<BV, TSZ, MODE, K>();
  static constexpr int PVS = PV | 1;  // padded-block stride of the centred codes (odd)
  static constexpr int XS = BV + 1;   // block stride of the values
  static constexpr int CS = BV + 8;   // block stride of the codes (16-byte rows for vector copies)
  static constexpr size_t a16(size_t v) { return (v + 15) & ~(size_t)15; }
  // fixed-point form: staged constants and B fragments
  static constexpr int QH = H1 == 32 ? 32 : 16;
  static constexpr size_t QB = MODE == 2 ? a16(sizeof(TcStage<QH>)) + a16(sizeof(WStage<QH>)) : 0;
  static constexpr size_t VP = sizeof(Tabs) + QB;
  static constexpr size_t X = VP + a16((size_t)GR * PVS * 4);
  static constexpr size_t L = X + a16((size_t)GR * XS * TSZ);
  static constexpr size_t C = L + a16((size_t)BV * 4);
  static constexpr size_t TOTAL = C + a16((size_t)GR * CS * 2);
};

template <int B0, int B1, int B2, int PV, int TSZ, int MODE, int K, int H1, int H2>
constexpr size_t recon_smem_bytes() {
  return ReconLayout<B0, B1, B2, PV, TSZ, MODE, K, H1, H2>::TOTAL;
}

// A coded point's value slot holds its code q until the waves are done.
template <typename T>
__device__ __forceinline__ void put_q(T* slot, int q) { *reinterpret_cast<int*>(slot) = q; }
template <typename T>
__device__ __forceinline__ int get_q(const T* slot) { return *reinterpret_cast<const int*>(slot); }

// Three CTAs per SM for the fixed-point form (80 registers, 73 KB of shared
// memory each): its waves are latency-bound, and more resident warps hide it.
template <typename T, int B0, int B1, int B2, int MODE, int K, int H1, int H2>
__global__ void __launch_bounds__(256, MODE == 1 ? 2 : 3) k_recon(Geo g, const uint8_t* __restrict__ in, DecInfo di, DecScratch ds,
                                               T* __restrict__ xo, const __grid_constant__ Mlp mlp,
                                               long long brick_lo, long long brick_hi) {
  constexpr int BV = B0 * B1 * B2;
  using BS = BrickShape<BV>;
  constexpr int G = BS::G, TS = BS::TS, NWT = TS / 32;
  constexpr int GR = recon_blocks<BV, (int)sizeof(T), MODE, K>(), NSUB = GR / G;  // blocks per brick, team groups
  constexpr bool WIDE = MODE != 0 && (K == 13 || K == 0);
  using PD = Pad<B0, B1, B2, WIDE>;
  using RL = ReconLayout<B0, B1, B2, PD::PV, (int)sizeof(T), MODE, K, H1, H2>;
  constexpr int PVS = RL::PVS, XS = RL::XS, CS = RL::CS;
  static_assert(sizeof(Tabs) % 16 == 0, "regions after the tables stay 16-byte aligned");
  constexpr int SZ = (B0 - 1) * 4 + (B1 - 1) * 2 + (B2 - 1) + 1;  // waves of the wider schedule
  constexpr int VW = 16 / (int)sizeof(T);
  constexpr bool VEC_OK = (B2 * GR) % VW == 0;
  extern __shared__ __align__(16) unsigned char smem[];
  Tabs& tb = *reinterpret_cast<Tabs*>(smem);
  constexpr int QK = MODE == 2 ? K : 7, QH = RL::QH;
  // fixed-point form only: constants and fragments
  TcStage<QH>& qst = *reinterpret_cast<TcStage<QH>*>(smem + sizeof(Tabs));
  WStage<QH>& qwf = *reinterpret_cast<WStage<QH>*>(smem + sizeof(Tabs) + RL::a16(sizeof(TcStage<QH>)));
  int* s_vp = reinterpret_cast<int*>(smem + RL::VP);             // GR padded blocks of centred codes
  T* s_x = reinterpret_cast<T*>(smem + RL::X);                    // GR blocks of values
  // BV points in wave order, each j | (padded index of j) << 16
  unsigned int* s_list = reinterpret_cast<unsigned int*>(smem + RL::L);
  uint16_t* s_cd = reinterpret_cast<uint16_t*>(smem + RL::C);     // GR blocks of codes
  __shared__ int s_ws[SZ + 2];
  __shared__ int s_fill[SZ + 2];
  __shared__ unsigned int s_wt[G][NWT];
  __shared__ int s_da[GR];
  __shared__ int s_bad;
  __shared__ int s_usen[GR], s_e2[GR];

  State c;
  c.Kp = di.Kp; c.Kn = di.Kn; c.Zq = di.Zq; c.S = di.S;
  if (sizeof(T) == 4) {
    c.step32 = __uint_as_float((unsigned int)di.step_bits);
    c.inv32 = __uint_as_float((unsigned int)di.inv_bits);
    c.ebdn32 = __uint_as_float((unsigned int)di.ebdn_bits);
  } else {
    c.stepd = __longlong_as_double((long long)di.step_bits);
    c.invd = __longlong_as_double((long long)di.inv_bits);
    c.ebdnd = __longlong_as_double((long long)di.ebdn_bits);
  }
  const int tid = threadIdx.x, lane = tid & 31;
  const bool s13 = di.stencil == 13;
  for (int i = tid; i < (int)(sizeof(Tabs) / 4); i += 256)
    reinterpret_cast<float*>(&tb)[i] = reinterpret_cast<const float*>(ds.ftab)[i];
  for (int i = tid; i < GR * PVS; i += 256) s_vp[i] = 0;
  for (int i = tid; i < SZ + 2; i += 256) { s_ws[i] = 0; s_fill[i] = 0; }
  if (tid == 0) s_bad = 0;
  if constexpr (MODE == 2) {
    tcnet_stage<QK, QH>(di.qnet, qst);
    wnet_stage<QK, QH>(di.qnet, qwf);
  }
  __syncthreads();
  for (int j = tid; j < BV; j += 256) {
    const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
    atomicAdd(&s_ws[(s13 ? 4 * lz + 2 * ly + lx : lz + ly + lx) + 1], 1);
  }
  __syncthreads();
  if (tid == 0)
    for (int i = 1; i < SZ + 2; ++i) s_ws[i] += s_ws[i - 1];
  __syncthreads();
  for (int j = tid; j < BV; j += 256) {
    const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
    const int sv = s13 ? 4 * lz + 2 * ly + lx : lz + ly + lx;
    s_list[s_ws[sv] + atomicAdd(&s_fill[sv], 1)] = (unsigned int)j | ((unsigned int)PD::at(lz, ly, lx) << 16);
  }
  const int nwave = s13 ? SZ : (B0 - 1) + (B1 - 1) + (B2 - 1) + 1;
  __syncthreads();
  if (*ds.err) return;
  const int R = 1 << (di.m - 1);
  const float sig = MODE ? __uint_as_float((unsigned int)(127 - mlp.s_in) << 23) : 1.0f;
  const float unsig = MODE ? __uint_as_float((unsigned int)(127 + mlp.s_in) << 23) : 1.0f;
  const T* ov = reinterpret_cast<const T*>(in + di.off_ov);
  const bool vec_rows = VEC_OK && (g.n[2] % VW == 0) && ((reinterpret_cast<uintptr_t>(xo) & 15u) == 0);
  const long long nbx = (g.nb[2] + GR - 1) / GR;
  const long long nbricks = g.nb[0] * g.nb[1] * nbx;
  const int team = tid / TS, t = tid % TS, wt = t >> 5;
  bool bad = false;
  (void)nbricks;
  for (long long brick = brick_lo + blockIdx.x; brick < brick_hi; brick += gridDim.x) {
    const long long bxg = brick % nbx;
    const long long byz = brick / nbx;
    const long long by = byz % g.nb[1];
    const long long bz = byz / g.nb[1];
    const long long z0 = bz * B0, y0 = by * B1, x0 = bxg * GR * B2;
    const int e0 = (int)min((long long)B0, g.n[0] - z0);
    const int e1 = (int)min((long long)B1, g.n[1] - y0);
    const int W = (int)min((long long)(GR * B2), g.n[2] - x0);
    // Each team sets up block team, team + G, ...; the per-team wave path
    // (one group) keeps its block's state below.
    bool bvalid = false, bfull = false, usen = false;
    int e2 = 0;
    int* vp = s_vp;
    T* xs = s_x;
    uint16_t* cd = s_cd;
    for (int sub = 0; sub < NSUB; ++sub) {
      const int blk = sub * G + team;
      const long long bx = bxg * GR + blk;
      bvalid = bx < g.nb[2];
      e2 = bvalid ? (int)min((long long)B2, g.n[2] - bx * B2) : 0;
      bfull = e0 == B0 && e1 == B1 && e2 == B2;
      const long long b = (bz * g.nb[1] + by) * g.nb[2] + bx;
      vp = s_vp + blk * PVS;
      xs = s_x + blk * XS;
      cd = s_cd + blk * CS;
      // codes (the decoder leaves positions in the codebook list, which maps
      // them to symbols) and the padded border for truncated blocks
      if (bvalid) {
        const uint4* src = reinterpret_cast<const uint4*>(ds.codes + b * BV);
        const uint16_t* __restrict__ sorted = ds.sorted;
        auto sym2 = [&](unsigned int u) {
          return (unsigned int)sorted[u & 0xFFFFu] | ((unsigned int)sorted[u >> 16] << 16);
        };
        for (int i = t; i < BV / 8; i += TS) {
          const uint4 v = src[i];
          reinterpret_cast<uint4*>(cd)[i] = make_uint4(sym2(v.x), sym2(v.y), sym2(v.z), sym2(v.w));
        }
        if (!bfull) {
          for (int j = t; j < BV; j += TS) {
            const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
            if (!(lz < e0 && ly < e1 && lx < e2)) vp[PD::at(lz, ly, lx)] = 0;
          }
        }
      }
      const unsigned int no = bvalid ? *reinterpret_cast<const uint16_t*>(in + di.off_bn + 2ull * b) : 1u;
      usen = bvalid && ((*reinterpret_cast<const unsigned int*>(in + di.off_bb + 4ull * b)) >> 31);
      const unsigned long long obase = bvalid ? ds.ooff[b] : 0ull;
      if (TS == 32) __syncwarp(); else __syncthreads();
      // balance points (code 0) per warp segment of the block
      constexpr int SEG = BV / NWT;  // contiguous codes per warp of the team
      unsigned int run = 0;
      if (bvalid) {
        for (int j0 = wt * SEG; j0 < (wt + 1) * SEG; j0 += 32) {
          const int j = j0 + lane;
          const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
          const bool f = j != 0 && (bfull || (lz < e0 && ly < e1 && lx < e2)) && cd[j] == 0;
          run += __popc(__ballot_sync(0xFFFFFFFFu, f));
        }
        if (NWT > 1 && lane == 0) s_wt[team][wt] = run;
      }
      // anchor: the block's first balance point (the container holds n_out >= nblocks of them)
      if (bvalid && t == 0) {
        const T xa = ov[obase < di.n_out ? obase : 0];
        bool okk;
        s_da[blk] = Num<T>::transform(xa, c, tb, okk);
        vp[PD::at(0, 0, 0)] = 0;
        xs[0] = xa;
      }
      if (t == 0) {
        s_usen[blk] = usen;
        s_e2[blk] = e2;
      }
      __syncthreads();
      unsigned int rank = 0, nzero = run;
      if (NWT > 1 && bvalid) {
        unsigned int tot = 0;
        for (int q = 0; q < NWT; ++q) {
          if (q < wt) rank += s_wt[team][q];
          tot += s_wt[team][q];
        }
        nzero = tot;
      }
      if (bvalid && (nzero + 1u != no || (usen && !MODE))) bad = true;
      // Every other balance point: its value and centred code go in before the
      // waves.  Only points of later waves read them.
      if (bvalid) {
        const int dab = s_da[blk];
        for (int j0 = wt * SEG; j0 < (wt + 1) * SEG; j0 += 32) {
          const int j = j0 + lane;
          const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
          const bool f = j != 0 && (bfull || (lz < e0 && ly < e1 && lx < e2)) && cd[j] == 0;
          const unsigned int bal = __ballot_sync(0xFFFFFFFFu, f);
          if (f) {
            const unsigned int r = 1u + rank + __popc(bal & ((1u << lane) - 1u));
            unsigned long long oi = obase + r;
            if (r >= no || oi >= di.n_out) { bad = true; oi = 0; }
            const T xv = ov[oi];
            bool okk;
            const int q = Num<T>::transform(xv, c, tb, okk);
            xs[j] = xv;
            vp[PD::at(lz, ly, lx)] = clampv((long long)q - dab);
          }
          rank += __popc(bal);
        }
      }
      __syncthreads();
    }
    const int da = s_da[team];  // the per-team path has one group: blk == team
    // Waves of all GR blocks at once: wave position f of the CTA is point
    // f / GR of the wave's list in block f % GR.
    const bool brick_full = e0 == B0 && e1 == B1 && W == GR * B2;
    if constexpr (MODE == 2) {
      // Each wave in tiles of 16 points through warp-level MMAs (a wave of a
      // few blocks is too narrow for 128-point tiles); the lanes of a quad
      // hold its two points' predictions.
      const int wid = tid >> 5, qc = lane & 3;
      int qoff[4];  // stencil offsets of this thread's input columns 2c, 2c + 1, 2c + 8, 2c + 9
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int col = 2 * qc + (i & 1) + 8 * (i >> 1);
        qoff[i] = col < QK ? PD::off(st_dz(QK, col), st_dy(QK, col), st_dx(QK, col)) : 0;
      }
      for (int sw = 1; sw < nwave; ++sw) {
        const int w0 = s_ws[sw], S = s_ws[sw + 1] - w0;
        const int tot = GR * S;
        // A wave's points read only earlier waves, so each tile finishes its own
        // points right after the network (lane c of a quad takes row g, lane
        // c + 1 row g + 8); one barrier per wave.
        for (int tile = wid; tile * 16 < tot; tile += 8) {
          int xv[2][4];
          int fs[2];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int f = tile * 16 + (lane >> 2) + 8 * r;
            fs[r] = f;
            const int fi = f < tot ? f : 0;
            const int pj = (fi % GR) * PVS + (int)(s_list[w0 + fi / GR] >> 16);
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[r][i] = s_vp[pj + qoff[i]];
          }
          int pq[2];
          wnet_tile<QK, QH>(qwf, qst, xv, pq[0], pq[1]);
          if (qc < 2) {
            const int f = fs[qc];
            if (f < tot) {
              const int gb = f % GR;
              const unsigned int e = s_list[w0 + f / GR];
              const int j = (int)(e & 0xFFFFu), pj = gb * PVS + (int)(e >> 16);
              bool valid = true;
              if (!brick_full) {
                const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
                valid = lz < e0 && ly < e1 && lx < s_e2[gb];
              }
              const unsigned int code = s_cd[gb * CS + j];
              if (valid && code != 0) {  // balance points are already in place
                long long prd;
                if (s_usen[gb]) {
                  prd = qc ? pq[1] : pq[0];
                } else {
                  int acc = 0;
#pragma unroll
                  for (int si = 0; si < 7; ++si)
                    acc += lz_w(7, si) * s_vp[pj + PD::off(s7_dz(si), s7_dy(si), s7_dx(si))];
                  prd = acc;
                }
                const int dag = s_da[gb];
                const long long qq = (long long)dag + prd + ((long long)code - R);
                int q;
                if (qq > 2147483647LL || qq < -2147483647LL) { bad = true; q = 0; }
                else q = (int)qq;
                put_q(&s_x[gb * XS + j], q);
                s_vp[pj] = clampv((long long)q - dag);
              }
            }
          }
        }
        __syncthreads();
      }
    } else if constexpr (MODE != 0 && K > 0) {
      // Two wave positions per thread through the packed perceptron forward.
      // Every neighbour load is unconditional (all indices are inside the
      // padded blocks), so a point's loads do not wait on its code.
      for (int sw = 1; sw < nwave; ++sw) {
        const int w0 = s_ws[sw], S = s_ws[sw + 1] - w0;
        const int tot = GR * S, half = (tot + 1) >> 1;
        for (int pr2 = tid; pr2 < half; pr2 += 256) {
          int inp[2][K];
          int pjs[2], xis[2], dav[2], lzp[2];
          unsigned int cds[2];
          bool act[2], need[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int f = pr2 + u * half;
            const int fi = f < tot ? f : 0;
            const int gb = fi % GR;
            const unsigned int e = s_list[w0 + fi / GR];
            const int j = (int)(e & 0xFFFFu), pj = gb * PVS + (int)(e >> 16);
            bool valid = f < tot;
            if (!brick_full) {
              const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
              valid = valid && lz < e0 && ly < e1 && lx < s_e2[gb];
            }
            const unsigned int code = s_cd[gb * CS + j];
            act[u] = valid && code != 0u;   // balance points are already in place
            need[u] = act[u] && s_usen[gb] != 0;
            cds[u] = code;
            pjs[u] = pj;
            xis[u] = gb * XS + j;
            dav[u] = s_da[gb];
#pragma unroll
            for (int si = 0; si < K; ++si) inp[u][si] = s_vp[pj + PD::off(st_dz(K, si), st_dy(K, si), st_dx(K, si))];
            int acc = 0;
#pragma unroll
            for (int si = 0; si < 7; ++si) acc += lz_w(7, si) * s_vp[pj + PD::off(s7_dz(si), s7_dy(si), s7_dx(si))];
            lzp[u] = acc;
          }
          float pv[2] = {0.0f, 0.0f};
          if (need[0] || need[1]) mlp_fwd2<K, H1, H2>(mlp, inp[0], inp[1], sig, unsig, pv[0], pv[1]);
          // both positions finish without branches, so their chains overlap
          int qv[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const long long prd = need[u] ? (long long)round_pred(pv[u]) : (long long)lzp[u];
            const long long qq = (long long)dav[u] + prd + ((long long)cds[u] - R);
            const bool ovf = qq > 2147483647LL || qq < -2147483647LL;
            bad |= act[u] && ovf;
            qv[u] = ovf ? 0 : (int)qq;
          }
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (act[u]) {
              put_q(&s_x[xis[u]], qv[u]);
              s_vp[pjs[u]] = clampv((long long)qv[u] - dav[u]);
            }
        }
        __syncthreads();
      }
    } else
    for (int sw = 1; sw < nwave; ++sw) {
      if (bvalid) {
        for (int idx = s_ws[sw] + t; idx < s_ws[sw + 1]; idx += TS) {
          const unsigned int e = s_list[idx];
          const int j = (int)(e & 0xFFFFu), pj = (int)(e >> 16);
          const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
          if (!bfull && !(lz < e0 && ly < e1 && lx < e2)) continue;
          const unsigned int code = cd[j];
          if (code == 0) continue;  // balance point, already in place
          long long pr = 0;
          bool done = false;
          if constexpr (MODE != 0) {
            if (usen) {
              constexpr int KK = K > 0 ? K : 13;
              int inp[KK];
              const int kk = K > 0 ? K : mlp.k;
#pragma unroll
              for (int si = 0; si < KK; ++si)
                inp[si] = si < kk ? vp[pj + PD::off(st_dz(kk, si), st_dy(kk, si), st_dx(kk, si))] : 0;
              float p;
              if constexpr (K > 0) p = mlp_fwd<K, H1, H2>(mlp, inp, sig, unsig);
              else p = mlp_fwd_rt(mlp, inp, sig, unsig);
              pr = round_pred(p);
              done = true;
            }
          }
          if (!done) {
            int acc = 0;
#pragma unroll
            for (int si = 0; si < 7; ++si) acc += lz_w(7, si) * vp[pj + PD::off(s7_dz(si), s7_dy(si), s7_dx(si))];
            pr = acc;
          }
          const long long qq = (long long)da + pr + ((long long)code - R);
          int q;
          if (qq > 2147483647LL || qq < -2147483647LL) { bad = true; q = 0; }
          else q = (int)qq;
          put_q(&xs[j], q);
          vp[pj] = clampv((long long)q - da);
        }
      }
      if (TS == 32) __syncwarp(); else __syncthreads();
    }
    __syncthreads();
    // The waves kept each coded point's code q in its value slot; the values
    // (the inverse map, Section III.B) need no wave order.
    for (int i = tid; i < GR * BV; i += 256) {
      const int gb = i / BV, j = i - gb * BV;
      if (j == 0) continue;  // the anchor holds its stored value
      const int lz = j / (B1 * B2), ly = (j / B2) % B1, lx = j % B2;
      if (!(lz < e0 && ly < e1 && lx < s_e2[gb])) continue;
      if (s_cd[gb * CS + j] == 0) continue;  // balance point: stored value
      T* slot = &s_x[gb * XS + j];
      *slot = Num<T>::recon(get_q(slot), c, tb);
    }
    __syncthreads();
    // coalesced brick store
    if (e0 == B0 && e1 == B1 && W == GR * B2 && vec_rows) {
      constexpr int RW = GR * B2 / VW;
      for (int e = tid; e < B0 * B1 * RW; e += 256) {
        const int r = e / RW, cv = e % RW;
        const int z = r / B1, y = r % B1;
        T v[VW];
#pragma unroll
        for (int q = 0; q < VW; ++q) {
          const int col = cv * VW + q;
          v[q] = s_x[(col / B2) * XS + (z * B1 + y) * B2 + (col % B2)];
        }
        uint4 u;
        memcpy(&u, v, 16);
        reinterpret_cast<uint4*>(xo + ((z0 + z) * g.n[1] + (y0 + y)) * g.n[2] + x0)[cv] = u;
      }
    } else {
      for (int e = tid; e < e0 * e1 * W; e += 256) {
        const int r = e / W, col = e - r * W;
        const int z = r / e1, y = r - z * e1;
        xo[((z0 + z) * g.n[1] + (y0 + y)) * g.n[2] + x0 + col] = s_x[(col / B2) * XS + (z * B1 + y) * B2 + (col % B2)];
      }
    }
    __syncthreads();
  }
  if (bad) s_bad = 1;
  __syncthreads();
  if (s_bad && tid == 0) atomicExch(ds.err, PC_ERR_CORRUPT);
}

template <typename T, int B0, int B1, int B2, int MODE, int K, int H1, int H2>
static int launch_r(const uint8_t* in, const Geo& g, const DecInfo& di, const DecScratch& ds, const Mlp& mlp, T* out,
                    int nsm, cudaStream_t s, SlabSink* sink) {
  constexpr int BV = B0 * B1 * B2;
  constexpr bool WIDE = MODE != 0 && (K == 13 || K == 0);
  auto kern = k_recon<T, B0, B1, B2, MODE, K, H1, H2>;
  constexpr size_t sm = recon_smem_bytes<B0, B1, B2, Pad<B0, B1, B2, WIDE>::PV, (int)sizeof(T), MODE, K, H1, H2>();
  static_assert(sm <= 232448, "shared memory per CTA");
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return PC_ERR_CUDA;
  if (MODE == 2 && cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return PC_ERR_CUDA;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
  if (per_sm < 1) per_sm = 1;
  constexpr int GR = recon_blocks<BV, (int)sizeof(T), MODE, K>();
  const long long nbricks = g.nb[0] * g.nb[1] * ((g.nb[2] + GR - 1) / GR);
  long long grid = (long long)nsm * per_sm;
  // With a host sink, the field goes out in slabs of whole block planes (z), each copied to the host on the
  // sink's stream while the next slab is reconstructed.
  const long long per_z = g.nb[1] * ((g.nb[2] + GR - 1) / GR);  // bricks per block plane
  const int nslab = (sink && B0 > 1 && g.nb[0] >= 2 * kSlabs) ? kSlabs : 1;
  ProfScope p(kStRecon, s);
  for (int k = 0; k < nslab; ++k) {
    const long long z0 = g.nb[0] * k / nslab, z1 = g.nb[0] * (k + 1) / nslab;
    const long long lo = nslab == 1 ? 0 : z0 * per_z, hi = nslab == 1 ? nbricks : z1 * per_z;
    long long gk = grid < hi - lo ? grid : hi - lo;
    if (gk < 1) gk = 1;
    kern<<<(unsigned int)gk, 256, sm, s>>>(g, in, di, ds, out, mlp, lo, hi);
    if (nslab > 1) {
      const size_t row = (size_t)g.n[1] * g.n[2] * sizeof(T);
      const size_t r0 = (size_t)(z0 * B0), r1 = (size_t)min((long long)g.n[0], z1 * B0);
      if (cudaEventRecord(sink->ev[k], s) != cudaSuccess || cudaStreamWaitEvent(sink->cs, sink->ev[k], 0) != cudaSuccess ||
          cudaMemcpyAsync(static_cast<uint8_t*>(sink->host) + r0 * row, reinterpret_cast<const uint8_t*>(out) + r0 * row,
                          (r1 - r0) * row, cudaMemcpyDeviceToHost, sink->cs) != cudaSuccess)
        return PC_ERR_CUDA;
    }
  }
  if (nslab > 1) {
    // the caller's stream waits for the last copy
    if (cudaEventRecord(sink->ev[kSlabs], sink->cs) != cudaSuccess ||
        cudaStreamWaitEvent(s, sink->ev[kSlabs], 0) != cudaSuccess)
      return PC_ERR_CUDA;
    sink->used = true;
  }
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

template <typename T, int B0, int B1, int B2>
static int launch_r_shape(const uint8_t* in, const Geo& g, const DecInfo& di, const DecScratch& ds, const Mlp& mlp,
                          T* out, int nsm, cudaStream_t s, SlabSink* sink) {
  if (!di.usenn_any) return launch_r<T, B0, B1, B2, 0, 0, 0, 0>(in, g, di, ds, mlp, out, nsm, s, sink);
  if (di.qmode) {
    if (mlp.k == 7 && mlp.h1 == 16 && mlp.h2 == 16)
      return launch_r<T, B0, B1, B2, 2, 7, 16, 16>(in, g, di, ds, mlp, out, nsm, s, sink);
    if (mlp.k == 13 && mlp.h1 == 32 && mlp.h2 == 32)
      return launch_r<T, B0, B1, B2, 2, 13, 32, 32>(in, g, di, ds, mlp, out, nsm, s, sink);
    return PC_ERR_ARG;
  }
  if (mlp.k == 7 && mlp.h1 == 16 && mlp.h2 == 16)
    return launch_r<T, B0, B1, B2, 1, 7, 16, 16>(in, g, di, ds, mlp, out, nsm, s, sink);
  if (mlp.k == 13 && mlp.h1 == 32 && mlp.h2 == 32)
    return launch_r<T, B0, B1, B2, 1, 13, 32, 32>(in, g, di, ds, mlp, out, nsm, s, sink);
  return launch_r<T, B0, B1, B2, 1, 0, 0, 0>(in, g, di, ds, mlp, out, nsm, s, sink);
}

// The fixed-point network read from the container must lie in its stated
// ranges (exact tensor-core sums, shifts inside 64 bits).
__global__ void k_qcheck(DecInfo di, int* err) {
  const int n = qnet_len(di.stencil, di.h1, di.h2);
  bool bad = false;
  if (threadIdx.x == 0) {
    // header: shapes, exponents, shifts (qnet_valid stops at the first entry check that fails)
    const long long* q = di.qnet;
    bad = q[0] != di.stencil || q[1] != di.h1 || q[2] != di.h2 || q[3] != di.s_in;
    for (int i = 4; i < 7; ++i) bad |= q[i] < -30 || q[i] > 30;
    for (int i = 7; i < 9; ++i) bad |= q[i] < 0 || q[i] > 26;
    const long long F = q[4] + q[5] + q[6] - q[7] - q[8];
    bad |= F < -20 || F > 62;
  }
  for (int i = kQHdr + threadIdx.x; i < n; i += blockDim.x)
    bad |= !qnet_entry_ok(di.qnet, i, di.stencil, di.h1, di.h2);
  if (bad) atomicExch(err, PC_ERR_CORRUPT);
}

template <typename T>
int launch_decompress(const uint8_t* in, const Geo& g, const DecInfo& di, const DecScratch& ds, const Mlp& mlp,
                      T* out, int nsm, cudaStream_t s, SlabSink* sink, int phase) {
  if (phase != kDecRecon) {
    if (di.qmode) k_qcheck<<<1, 256, 0, s>>>(di, ds.err);
    { ProfScope p(kStDecTables, s); k_dec_tables<<<1, 1024, 0, s>>>(in, di, ds); }
    const unsigned int nc = (unsigned int)g.nchunks;
    {
      ProfScope p(kStDecScan, s);
      k_dec_chunksum<<<nc, 256, 0, s>>>(g, in, di, ds);
      k_dec_chunkscan<<<1, 1024, 0, s>>>(g, di, ds);
      k_dec_blockoff<<<nc, 256, 0, s>>>(g, in, di, ds);
    }
    if (phase == kDecPrep) return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
    {
      ProfScope p(kStHuffDecode, s);
      k_huff_decode<<<(unsigned int)((g.nblocks + kDecThreads - 1) / kDecThreads), kDecThreads, 0, s>>>(g, in, di,
                                                                                                       ds);
    }
    if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  }
  if (di.literal) {
    if constexpr (sizeof(T) == 4) return launch_lit_decode(in, g, di, ds, mlp, out, nsm, s);
    return PC_ERR_ARG;
  }
  const int b0 = g.b[0], b1 = g.b[1], b2 = g.b[2];
#define PC_SHAPE(A, B, C) \
  if (b0 == A && b1 == B && b2 == C) return launch_r_shape<T, A, B, C>(in, g, di, ds, mlp, out, nsm, s, sink);
  PC_SHAPE(8, 8, 8)
  PC_SHAPE(4, 4, 4)
  PC_SHAPE(16, 16, 16)
  PC_SHAPE(1, 16, 32)
  PC_SHAPE(1, 8, 8)
  PC_SHAPE(1, 64, 64)
#undef PC_SHAPE
  return PC_ERR_ARG;
}
template int launch_decompress<float>(const uint8_t*, const Geo&, const DecInfo&, const DecScratch&, const Mlp&,
                                      float*, int, cudaStream_t, SlabSink*, int);
template int launch_decompress<double>(const uint8_t*, const Geo&, const DecInfo&, const DecScratch&, const Mlp&,
                                       double*, int, cudaStream_t, SlabSink*, int);

}  // namespace pc
