// a11-a12: per-block code-length sums, their prefix scan, the container
// header, and bit-packing of the code words and balance points.
//
// Blocks are grouped in chunks of about 16K points.  k_blockbits sums each
// block's code lengths and writes the block table; k_chunkscan scans the chunk
// totals in one CTA, fixes the section offsets, writes the header (with its
// CRC-32) and the weights, and zeroes the stream words that two chunks share;
// k_pack assembles each chunk's bits in shared memory (code words MSB first)
// and writes whole words, using atomicOr only on the two boundary words.
#include "pc_kernels.cuh"
#include "pc_profile.cuh"

namespace pc {

__device__ __forceinline__ void block_coords(const Geo& g, long long b, long long& bz, long long& by, long long& bx,
                                             int& e0, int& e1, int& e2) {
  bx = b % g.nb[2];
  const long long t = b / g.nb[2];
  by = t % g.nb[1];
  bz = t / g.nb[1];
  e0 = (int)min((long long)g.b[0], g.n[0] - bz * g.b[0]);
  e1 = (int)min((long long)g.b[1], g.n[1] - by * g.b[1]);
  e2 = (int)min((long long)g.b[2], g.n[2] - bx * g.b[2]);
}

// padded raster index j of a block -> does it hold a non-anchor point?
__device__ __forceinline__ bool slot_valid(const Geo& g, int j, int e0, int e1, int e2, bool full) {
  if (j == 0) return false;
  if (full) return true;
  const int b12 = g.b[1] * g.b[2];
  const int lz = j / b12, r = j - lz * b12, ly = r / g.b[2], lx = r - ly * g.b[2];
  return lz < e0 && ly < e1 && lx < e2;
}

__global__ void __launch_bounds__(256) k_blockbits(Geo g, const uint16_t* __restrict__ codes,
                                                   const uint8_t* __restrict__ nnflag,
                                                   const uint32_t* __restrict__ nout, const uint8_t* __restrict__ lens,
                                                   uint32_t* __restrict__ bbits, unsigned long long* chunk_bits,
                                                   unsigned long long* chunk_nout, const State* __restrict__ st,
                                                   uint8_t* out) {
  __shared__ unsigned long long s_b[8], s_o[8];
  if (st->err) return;
  const long long c = blockIdx.x;
  const long long b0 = c * g.ch, b1 = min(g.nblocks, b0 + g.ch);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned long long off_bb = st->off_bb, off_bn = st->off_bn;
  unsigned long long wb = 0, wo = 0;
  for (long long b = b0 + wid; b < b1; b += 8) {
    long long bz, by, bx;
    int e0, e1, e2;
    block_coords(g, b, bz, by, bx, e0, e1, e2);
    const bool full = e0 == g.b[0] && e1 == g.b[1] && e2 == g.b[2];
    unsigned int s = 0;
    const uint16_t* cb = codes + b * g.bvol;
    if (full && (g.bvol & 255) == 0) {
      for (int j8 = lane; j8 < g.bvol / 8; j8 += 32) {
        const uint4 v = *reinterpret_cast<const uint4*>(cb + 8 * j8);
        const unsigned int u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 8 * j8 + 2 * q;
          s += (j != 0 ? lens[u[q] & 0xFFFFu] : 0u) + lens[u[q] >> 16];
        }
      }
    } else {
      for (int j = lane; j < g.bvol; j += 32)
        if (slot_valid(g, j, e0, e1, e2, full)) s += lens[cb[j]];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) {
      bbits[b] = s;
      const unsigned int no = nout[b];
      st_u32(out + off_bb + 4ull * b, s | ((unsigned int)nnflag[b] << 31));
      *reinterpret_cast<uint16_t*>(out + off_bn + 2ull * b) = (uint16_t)no;
      wb += s;
      wo += no;
    }
  }
  if (lane == 0) { s_b[wid] = wb; s_o[wid] = wo; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tb = 0, to = 0;
    for (int i = 0; i < 8; ++i) { tb += s_b[i]; to += s_o[i]; }
    chunk_bits[c] = tb;
    chunk_nout[c] = to;
  }
}


// The 256-byte header, assembled in shared memory (s_hdr) by the whole CTA
// and checksummed there (CRC-32, reflected 0xEDB88320, table in s_crc);
// the caller copies it out.  Contains __syncthreads.
template <typename T>
__device__ void write_header(uint8_t* s_hdr, unsigned int* s_crc, const State& c, const Geo& g, const HdrInfo& hi,
                             unsigned long long to, unsigned long long swords, unsigned long long off_bb,
                             unsigned long long off_bn, unsigned long long off_ov, unsigned long long off_st,
                             unsigned long long total) {
  const int tid = threadIdx.x;
  if (tid < 256) {
    unsigned int cr = (unsigned int)tid;
    for (int k = 0; k < 8; ++k) cr = (cr >> 1) ^ (0xEDB88320u & (0u - (cr & 1u)));
    s_crc[tid] = cr;
  }
  if (tid < 64) st_u32(s_hdr + 4 * tid, 0u);
  __syncthreads();
  if (tid == 0) {
    uint8_t* const hd = s_hdr;
    const bool nn = hi.pred != 0;
    st_u32(hd + 0, 0x504D4350u);  // "PCMP"
    st_u32(hd + 4, 1u);
    st_u32(hd + 8, (unsigned int)hi.dtype);
    st_u32(hd + 12, (unsigned int)hi.pred);
    st_u64(hd + 16, (unsigned long long)g.n[0]);
    st_u64(hd + 24, (unsigned long long)g.n[1]);
    st_u64(hd + 32, (unsigned long long)g.n[2]);
    st_u32(hd + 40, (unsigned int)g.b[0]);
    st_u32(hd + 44, (unsigned int)g.b[1]);
    st_u32(hd + 48, (unsigned int)g.b[2]);
    st_u32(hd + 52, nn ? (unsigned int)hi.stencil : 0u);
    st_u32(hd + 56, nn ? (unsigned int)hi.h1 : 0u);
    st_u32(hd + 60, nn ? (unsigned int)hi.h2 : 0u);
    st_u32(hd + 64, (unsigned int)hi.m);
    st_u32(hd + 68, nn ? (unsigned int)hi.s_in : 0u);
    st_u64(hd + 72, (unsigned long long)__double_as_longlong(hi.eb));
    st_u64(hd + 80, (unsigned long long)__double_as_longlong(c.amin));
    st_u64(hd + 88, (unsigned long long)__double_as_longlong(c.amax));
    st_u32(hd + 96, (unsigned int)c.trivial);
    st_u32(hd + 100, (unsigned int)c.Kp);
    st_u32(hd + 104, (unsigned int)c.Kn);
    st_u32(hd + 108, (unsigned int)c.Zq);
    st_u32(hd + 112, (unsigned int)c.S);
    st_u32(hd + 116, c.n_used);
    if (sizeof(T) == 4) {
      st_u64(hd + 120, __float_as_uint(c.step32));
      st_u64(hd + 128, __float_as_uint(c.inv32));
      st_u64(hd + 136, __float_as_uint(c.ebdn32));
    } else {
      st_u64(hd + 120, (unsigned long long)__double_as_longlong(c.stepd));
      st_u64(hd + 128, (unsigned long long)__double_as_longlong(c.invd));
      st_u64(hd + 136, (unsigned long long)__double_as_longlong(c.ebdnd));
    }
    st_u64(hd + 144, (unsigned long long)g.nblocks);
    st_u64(hd + 152, to);
    st_u64(hd + 160, swords);
    st_u64(hd + 168, (unsigned long long)kHdr);
    st_u64(hd + 176, hi.off_cb);
    st_u64(hd + 184, off_bb);
    st_u64(hd + 192, off_bn);
    st_u64(hd + 200, off_ov);
    st_u64(hd + 208, off_st);
    st_u64(hd + 216, total);
    st_u32(hd + 224, (unsigned int)hi.nw);
    st_u32(hd + 228, hi.flags);
    st_u32(hd + 232, (unsigned int)hi.eq_period);
    unsigned int crc = 0xFFFFFFFFu;
    for (int i = 0; i < 252; ++i) crc = s_crc[(crc ^ hd[i]) & 0xFFu] ^ (crc >> 8);
    st_u32(hd + 252, crc ^ 0xFFFFFFFFu);
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(1024) k_chunkscan(Geo g, const unsigned long long* __restrict__ chunk_bits,
                                                    const unsigned long long* __restrict__ chunk_nout,
                                                    unsigned long long* chunk_boff, unsigned long long* chunk_ooff,
                                                    State* st, uint8_t* out, HdrInfo hi,
                                                    const __grid_constant__ Mlp mlp) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned int s_crc[256];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (st->err) return;
  const long long nc = g.nchunks;
  const long long per = (nc + nt - 1) / nt;
  const long long lo = min(nc, tid * per), hi2 = min(nc, lo + per);
  unsigned long long sb = 0, so = 0;
  for (long long i = lo; i < hi2; ++i) { sb += chunk_bits[i]; so += chunk_nout[i]; }
  unsigned long long tb, to;
  unsigned long long pb = cta_exscan<unsigned long long>(sb, s_w, tb);
  unsigned long long po = cta_exscan<unsigned long long>(so, s_w, to);
  for (long long i = lo; i < hi2; ++i) {
    chunk_boff[i] = pb;
    chunk_ooff[i] = po;
    pb += chunk_bits[i];
    po += chunk_nout[i];
  }
  const unsigned long long ts = sizeof(T);
  const unsigned long long swords = (tb + 31) / 32;
  const unsigned long long off_bb = st->off_bb, off_bn = st->off_bn;
  const unsigned long long off_ov = al16(off_bn + 2ull * (unsigned long long)g.nblocks);
  const unsigned long long off_st = al16(off_ov + ts * to);
  const unsigned long long total = al16(off_st + 4ull * swords);
  __syncthreads();
  if (total > hi.cap) {
    if (tid == 0) st->err = PC_ERR_CAPACITY;
    return;
  }
  if (tid == 0) {
    st->n_out = to;
    st->total_bits = tb;
    st->swords = swords;
    st->off_ov = off_ov;
    st->off_st = off_st;
    st->total = total;
    st->out_size = total;
  }
  // zero the stream words shared between chunks, the section pads and the stream tail
  uint32_t* stream = reinterpret_cast<uint32_t*>(out + off_st);
  for (long long i = lo; i < hi2; ++i) {
    const unsigned long long bits = chunk_bits[i];
    if (bits) {
      const unsigned long long s0 = chunk_boff[i];
      stream[s0 >> 5] = 0u;
      stream[(s0 + bits - 1) >> 5] = 0u;
    }
  }
  for (unsigned long long i = off_bb + 4ull * g.nblocks + tid; i < off_bn; i += nt) out[i] = 0;
  for (unsigned long long i = off_bn + 2ull * g.nblocks + tid; i < off_ov; i += nt) out[i] = 0;
  for (unsigned long long i = off_ov + ts * to + tid; i < off_st; i += nt) out[i] = 0;
  for (unsigned long long i = off_st + 4ull * swords + tid; i < total; i += nt) out[i] = 0;
  // weights and their pad
  // the f32 weights; the fixed-point network was placed there by the host
  if (hi.pred == 1)
    for (int i = tid; i < hi.nw; i += nt) st_u32(out + kHdr + 4ull * i, __float_as_uint(mlp.w[i]));
  for (unsigned long long i = kHdr + (unsigned long long)hi.wsz * hi.nw + tid; i < hi.off_cb; i += nt) out[i] = 0;
  // header
  __shared__ __align__(16) uint8_t s_hdr[256];
  write_header<T>(s_hdr, s_crc, *st, g, hi, to, swords, off_bb, off_bn, off_ov, off_st, total);
  if (tid < 64) st_u32(out + 4 * tid, reinterpret_cast<const unsigned int*>(s_hdr)[tid]);
}

// ---------------------------------------------------------------------------
// Finish of a single-pass compression (the sample codebook of the training
// phase, Section IV.C).  The last brick's inclusive prefixes give the stream
// bits and balance points; the stream ends the fixed sections and the balance
// values follow it.  Each stream word that several bricks share is assembled
// by the brick holding its first bit, from the edge words the bricks kept
// aside; the balance values move from the workspace to their section; CTA 0
// writes the pads, the weights and the header.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sp_finish(Geo g, State* st, uint8_t* out, HdrInfo hi,
                                                   const __grid_constant__ Mlp mlp, SpFinish f) {
  __shared__ unsigned int s_crc[256];
  __shared__ __align__(16) uint8_t s_hdr[256];
  if (st->err) return;
  constexpr unsigned long long kV = (1ull << 62) - 1;
  const unsigned long long* rb = f.rec;
  const unsigned long long* ro = f.rec + f.nbk;
  const unsigned long long tb = rb[f.nbk - 1] & kV, to = ro[f.nbk - 1] & kV;
  const unsigned long long ts = sizeof(T);
  const unsigned long long swords = (tb + 31) / 32;
  const unsigned long long off_st = f.off_st;
  const unsigned long long off_ov = al16(off_st + 4ull * swords);
  const unsigned long long total = al16(off_ov + ts * to);
  const int tid = threadIdx.x;
  if (total > hi.cap) {
    if (blockIdx.x == 0 && tid == 0) st->err = PC_ERR_CAPACITY;
    return;
  }
  const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + tid;
  const unsigned long long gs = (unsigned long long)gridDim.x * blockDim.x;
  uint32_t* stream = reinterpret_cast<uint32_t*>(out + off_st);
  for (unsigned long long k = gt; k < (unsigned long long)f.nbk; k += gs) {
    const unsigned long long sk = k ? (rb[k - 1] & kV) : 0ull;
    const unsigned long long ek = rb[k] & kV;
    if (ek == sk || (ek & 31ull) == 0ull) continue;  // no bits, or the last word is whole
    const unsigned long long lw = (ek - 1) >> 5;
    if (sk > 32ull * lw) continue;  // the word's first bit is an earlier brick's
    unsigned int v = (sk >> 5) == lw ? f.side[2 * k] : f.side[2 * k + 1];
    for (unsigned long long j = k + 1; j < (unsigned long long)f.nbk; ++j) {
      const unsigned long long sj = rb[j - 1] & kV;
      if (sj >= 32ull * (lw + 1)) break;
      if ((rb[j] & kV) > sj) v |= f.side[2 * j];
    }
    stream[lw] = v;
  }
  const T* ovs = static_cast<const T*>(f.ov);
  T* ovd = reinterpret_cast<T*>(out + off_ov);
  for (unsigned long long i = gt; i < to; i += gs) ovd[i] = ovs[i];
  if (blockIdx.x != 0) return;
  const int nt = blockDim.x;
  if (tid == 0) {
    st->n_out = to;
    st->total_bits = tb;
    st->swords = swords;
    st->off_ov = off_ov;
    st->off_st = off_st;
    st->total = total;
    st->out_size = total;
  }
  const unsigned long long off_bb = f.off_bb, off_bn = f.off_bn;
  for (unsigned long long i = hi.off_cb + 4ull * st->n_used + tid; i < off_bb; i += nt) out[i] = 0;
  for (unsigned long long i = off_bb + 4ull * g.nblocks + tid; i < off_bn; i += nt) out[i] = 0;
  for (unsigned long long i = off_bn + 2ull * g.nblocks + tid; i < off_st; i += nt) out[i] = 0;
  for (unsigned long long i = off_st + 4ull * swords + tid; i < off_ov; i += nt) out[i] = 0;
  for (unsigned long long i = off_ov + ts * to + tid; i < total; i += nt) out[i] = 0;
  if (hi.pred == 1)
    for (int i = tid; i < hi.nw; i += nt) st_u32(out + kHdr + 4ull * i, __float_as_uint(mlp.w[i]));
  for (unsigned long long i = kHdr + (unsigned long long)hi.wsz * hi.nw + tid; i < hi.off_cb; i += nt) out[i] = 0;
  write_header<T>(s_hdr, s_crc, *st, g, hi, to, swords, off_bb, off_bn, off_ov, off_st, total);
  if (tid < 64) st_u32(out + 4 * tid, reinterpret_cast<const unsigned int*>(s_hdr)[tid]);
}

template <typename T>
int launch_sp_finish(const Geo& g, State* st, uint8_t* out, const HdrInfo& hi, const Mlp& mlp, const SpFinish& f,
                     int nsm, cudaStream_t s) {
  ProfScope p(kStPack, s);
  k_sp_finish<T><<<(unsigned int)nsm, 256, 0, s>>>(g, st, out, hi, mlp, f);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
template int launch_sp_finish<float>(const Geo&, State*, uint8_t*, const HdrInfo&, const Mlp&, const SpFinish&, int,
                                     cudaStream_t);
template int launch_sp_finish<double>(const Geo&, State*, uint8_t*, const HdrInfo&, const Mlp&, const SpFinish&, int,
                                      cudaStream_t);

template <typename T>
__global__ void __launch_bounds__(256) k_pack(Geo g, const T* __restrict__ x, const uint16_t* __restrict__ codes,
                                              const uint32_t* __restrict__ nout, const uint32_t* __restrict__ bbits,
                                              const uint32_t* __restrict__ cwl,
                                              const unsigned long long* __restrict__ chunk_bits,
                                              const unsigned long long* __restrict__ chunk_boff,
                                              const unsigned long long* __restrict__ chunk_ooff,
                                              const State* __restrict__ st, uint8_t* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int s_w[32];
  if (st->err) return;
  const long long c = blockIdx.x;
  const long long b0 = c * g.ch, b1 = min(g.nblocks, b0 + g.ch);
  const int nb = (int)(b1 - b0);
  unsigned int* s_boff = reinterpret_cast<unsigned int*>(smem);    // [ch]
  unsigned int* s_ooff = s_boff + g.ch;                            // [ch]
  unsigned int* s_words = s_ooff + g.ch;                           // chunk bit buffer
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // per-block offsets inside the chunk
  const int per = (nb + 255) / 256;
  const int lo = min(nb, tid * per), hi = min(nb, lo + per);
  unsigned int sb = 0, so = 0;
  for (int i = lo; i < hi; ++i) { sb += bbits[b0 + i]; so += nout[b0 + i]; }
  unsigned int tb, to;
  unsigned int pb = cta_exscan<unsigned int>(sb, s_w, tb);
  unsigned int po = cta_exscan<unsigned int>(so, s_w, to);
  for (int i = lo; i < hi; ++i) {
    s_boff[i] = pb;
    s_ooff[i] = po;
    pb += bbits[b0 + i];
    po += nout[b0 + i];
  }
  const unsigned long long S = chunk_boff[c];
  const unsigned long long CB = chunk_bits[c];
  const int sh = (int)(S & 31ull);
  const int nwords = (int)((sh + CB + 31) >> 5);
  for (int i = tid; i < nwords; i += 256) s_words[i] = 0u;
  __syncthreads();
  const unsigned long long off_ov = st->off_ov, off_st = st->off_st;
  T* ov = reinterpret_cast<T*>(out + off_ov);
  const unsigned long long obase = chunk_ooff[c];
  const int b12 = g.b[1] * g.b[2];
  for (int i = wid; i < nb; i += 8) {
    const long long b = b0 + i;
    long long bz, by, bx;
    int e0, e1, e2;
    block_coords(g, b, bz, by, bx, e0, e1, e2);
    const bool full = e0 == g.b[0] && e1 == g.b[1] && e2 == g.b[2];
    const long long z0 = bz * g.b[0], y0 = by * g.b[1], x0 = bx * g.b[2];
    unsigned int pos = (unsigned int)sh + s_boff[i];
    unsigned long long op = obase + s_ooff[i];
    if (lane == 0) ov[op] = x[(z0 * g.n[1] + y0) * g.n[2] + x0];
    op += 1;
    const uint16_t* cb = codes + b * g.bvol;
    // each lane packs 8 consecutive codes (one 16-byte load)
    for (int j0 = 0; j0 < g.bvol; j0 += 256) {
      const int jl = j0 + 8 * lane;
      unsigned int cd[8];
      if (jl + 8 <= g.bvol) {
        const uint4 v = *reinterpret_cast<const uint4*>(cb + jl);
        cd[0] = v.x & 0xFFFFu; cd[1] = v.x >> 16; cd[2] = v.y & 0xFFFFu; cd[3] = v.y >> 16;
        cd[4] = v.z & 0xFFFFu; cd[5] = v.z >> 16; cd[6] = v.w & 0xFFFFu; cd[7] = v.w >> 16;
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) cd[q] = 0u;
      }
      unsigned int ent[8];
      unsigned int lbits = 0, louts = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = jl + q;
        const bool valid = j < g.bvol && slot_valid(g, j, e0, e1, e2, full);
        ent[q] = valid ? cwl[cd[q]] : 0u;   // (length << 24) | code word
        lbits += ent[q] >> 24;
        louts += (valid && cd[q] == 0u) ? 1u : 0u;
      }
      unsigned int ib = lbits, io = louts;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int yb = __shfl_up_sync(0xFFFFFFFFu, ib, o);
        const unsigned int yo = __shfl_up_sync(0xFFFFFFFFu, io, o);
        if (lane >= o) { ib += yb; io += yo; }
      }
      unsigned int p = pos + ib - lbits;
      unsigned long long o2 = op + (io - louts);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const unsigned int L = ent[q] >> 24, wv = ent[q] & 0xFFFFFFu;
        if (L) {
          const unsigned int wi = p >> 5, bo = p & 31u;
          if (bo + L <= 32u) {
            atomicOr(&s_words[wi], wv << (32u - bo - L));
          } else {
            atomicOr(&s_words[wi], wv >> (bo + L - 32u));
            atomicOr(&s_words[wi + 1], wv << (64u - bo - L));
          }
          p += L;
        }
        const int j = jl + q;
        if (j < g.bvol && cd[q] == 0u && slot_valid(g, j, e0, e1, e2, full)) {
          const int lz = j / b12, r = j - lz * b12, ly = r / g.b[2], lx = r - ly * g.b[2];
          ov[o2] = x[((z0 + lz) * g.n[1] + (y0 + ly)) * g.n[2] + x0 + lx];
          ++o2;
        }
      }
      pos += __shfl_sync(0xFFFFFFFFu, ib, 31);
      op += __shfl_sync(0xFFFFFFFFu, io, 31);
    }
  }
  __syncthreads();
  if (CB == 0) return;
  uint32_t* stream = reinterpret_cast<uint32_t*>(out + off_st);
  const unsigned long long W0 = S >> 5;
  for (int wi = tid; wi < nwords; wi += 256) {
    const unsigned long long gw = W0 + wi;
    const bool inside = gw * 32ull >= S && gw * 32ull + 32ull <= S + CB;
    if (inside) stream[gw] = s_words[wi];
    else atomicOr(&stream[gw], s_words[wi]);
  }
}

template <typename T>
int launch_pack(const T* x, const Geo& g, const uint16_t* codes, const uint8_t* nnflag, const uint32_t* nout,
                const uint8_t* lens, const uint32_t* cw, uint32_t* bbits, unsigned long long* chunk_bits,
                unsigned long long* chunk_nout, unsigned long long* chunk_boff, unsigned long long* chunk_ooff,
                State* st, uint8_t* out, const HdrInfo& hi, const Mlp& mlp, cudaStream_t s) {
  const unsigned int nc = (unsigned int)g.nchunks;
  { ProfScope p(kStBlockbits, s); k_blockbits<<<nc, 256, 0, s>>>(g, codes, nnflag, nout, lens, bbits, chunk_bits, chunk_nout, st, out); }
  { ProfScope p(kStChunkscan, s); k_chunkscan<T><<<1, 1024, 0, s>>>(g, chunk_bits, chunk_nout, chunk_boff, chunk_ooff, st, out, hi, mlp); }
  const size_t words = ((size_t)g.ch * (size_t)(g.bvol > 1 ? g.bvol - 1 : 1) * kLmax + 31) / 32 + 2;
  const size_t smem = (size_t)g.ch * 8 + words * 4;
  if (cudaFuncSetAttribute(k_pack<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PC_ERR_CUDA;
  { ProfScope p(kStPack, s); k_pack<T><<<nc, 256, smem, s>>>(g, x, codes, nout, bbits, cw, chunk_bits, chunk_boff, chunk_ooff, st, out); }
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
template int launch_pack<float>(const float*, const Geo&, const uint16_t*, const uint8_t*, const uint32_t*,
                                const uint8_t*, const uint32_t*, uint32_t*, unsigned long long*, unsigned long long*,
                                unsigned long long*, unsigned long long*, State*, uint8_t*, const HdrInfo&, const Mlp&,
                                cudaStream_t);
template int launch_pack<double>(const double*, const Geo&, const uint16_t*, const uint8_t*, const uint32_t*,
                                 const uint8_t*, const uint32_t*, uint32_t*, unsigned long long*, unsigned long long*,
                                 unsigned long long*, unsigned long long*, State*, uint8_t*, const HdrInfo&,
                                 const Mlp&, cudaStream_t);

}  // namespace pc
