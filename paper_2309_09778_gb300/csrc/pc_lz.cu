// The fourth SZ stage (Section IV.A): a lossless pass over the bitstream
// bytes, which the paper names and Algorithm 1 leaves out.  An LZ77-style
// matcher over independent chunks of kLzChunk bytes, one thread per chunk:
//   - tokens: a control byte c < 128 is followed by c + 1 literal bytes; a
//     control byte c >= 128 is a match of (c - 128) + 4 bytes (4..131) at a
//     distance d (1..chunk) given by the next two bytes, little-endian;
//   - greedy parse: at position i (4 bytes left) the hash of the 4 bytes at i,
//     (b0 | b1 << 8 | b2 << 16 | b3 << 24) * 2654435761 >> 20 (Knuth's
//     multiplicative hashing), names the last position that started a parse
//     step with that hash; 4 or more matching bytes there give the longest
//     match up to 131 bytes, else one literal; the table then names i;
//     literals go out in runs of up to 128 before the next match or the end;
//   - a chunk whose tokens are not shorter than itself is stored as is.
// Section: u32 chunk count, u32 chunk bytes, u64 raw bytes, then per chunk
// u32 (coded bytes | stored << 31), 16-byte aligned, then the chunks' bytes
// back to back.
#include "pc_kernels.cuh"
#include "pc_profile.cuh"

namespace pc {

constexpr int kLzHashBits = 12;

__device__ __forceinline__ unsigned int lz_hash(const uint8_t* p) {
  const unsigned int v = (unsigned int)p[0] | ((unsigned int)p[1] << 8) | ((unsigned int)p[2] << 16) |
                         ((unsigned int)p[3] << 24);
  return (v * 2654435761u) >> (32 - kLzHashBits);
}

__device__ __forceinline__ unsigned int lz_lits(const uint8_t* src, unsigned int a, unsigned int b, uint8_t* dst,
                                                unsigned int o) {
  while (a < b) {
    const unsigned int r = b - a < 128u ? b - a : 128u;
    dst[o++] = (uint8_t)(r - 1);
    for (unsigned int k = 0; k < r; ++k) dst[o++] = src[a + k];
    a += r;
  }
  return o;
}

// One warp per chunk (grid over the most chunks a stream of this field can
// have; the stream's length is on the device).  The warp stages the chunk and
// a fresh hash table in shared memory; lane 0 runs the greedy parse (serial by
// nature) against them and writes the tokens to the chunk's slot; the warp
// then writes the raw chunk instead when the tokens are not shorter.  Sizes:
// coded bytes | stored << 31.
constexpr int kLzWarps = 4;
__global__ void __launch_bounds__(32 * kLzWarps) k_lz_encode(const uint8_t* __restrict__ out, unsigned long long nch_max,
                                                             uint8_t* slots, unsigned int* sizes,
                                                             const State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char lzsm[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* sdat = lzsm + (size_t)wid * (kLzChunk + 2 * (1 << kLzHashBits));
  uint16_t* tab = reinterpret_cast<uint16_t*>(sdat + kLzChunk);
  const unsigned long long c = (unsigned long long)blockIdx.x * kLzWarps + wid;
  if (c >= nch_max || st->err) return;
  const unsigned long long nraw = 4ull * st->swords;
  if (c * kLzChunk >= nraw) return;
  const uint8_t* src = out + st->off_st + c * kLzChunk;
  const unsigned int n = (unsigned int)(nraw - c * kLzChunk < (unsigned long long)kLzChunk ? nraw - c * kLzChunk
                                                                                            : kLzChunk);
  // the chunk (16-byte loads: the stream starts 16-byte aligned, chunks are 16 KiB, n a multiple of 4)
  for (unsigned int i = 4 * lane; i < n; i += 128) *reinterpret_cast<unsigned int*>(sdat + i) =
      *reinterpret_cast<const unsigned int*>(src + i);
  for (int i = lane; i < (1 << kLzHashBits) / 2; i += 32) reinterpret_cast<unsigned int*>(tab)[i] = 0u;
  __syncwarp();
  uint8_t* dst = slots + c * kLzSlot;
  unsigned int o = 0;
  if (lane == 0) {
    unsigned int i = 0, lit0 = 0;
    while (i < n) {
      unsigned int L = 0, d = 0;
      if (i + 4 <= n) {
        const unsigned int h = lz_hash(sdat + i);
        const unsigned int cand = tab[h];
        tab[h] = (uint16_t)(i + 1);
        if (cand) {
          const unsigned int j = cand - 1;
          while (i + L < n && L < 131u && sdat[j + L] == sdat[i + L]) ++L;
          if (L >= 4) d = i - j;
          else L = 0;
        }
      }
      if (L) {
        o = lz_lits(sdat, lit0, i, dst, o);
        dst[o++] = (uint8_t)(128 + (L - 4));
        dst[o++] = (uint8_t)(d & 0xFFu);
        dst[o++] = (uint8_t)(d >> 8);
        i += L;
        lit0 = i;
      } else {
        ++i;
      }
      if (o >= n) break;  // no shorter than the chunk: it is stored
    }
    if (o < n) o = lz_lits(sdat, lit0, n, dst, o);
  }
  o = __shfl_sync(0xFFFFFFFFu, o, 0);
  if (o >= n) {
    for (unsigned int i = 4 * lane; i < n; i += 128)
      *reinterpret_cast<unsigned int*>(dst + i) = *reinterpret_cast<const unsigned int*>(sdat + i);
    if (lane == 0) sizes[c] = n | 0x80000000u;
  } else if (lane == 0) {
    sizes[c] = o;
  }
}

// One CTA: section offsets of the chunks, the section's header and table, the
// container's new size; the header (size, flag, section bytes, CRC) rewritten.
__global__ void __launch_bounds__(1024) k_lz_layout(const unsigned int* __restrict__ sizes, unsigned long long* offs,
                                                    State* st, uint8_t* out, unsigned long long cap) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned int s_crc[256];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (st->err) return;
  const unsigned long long off_st = st->off_st;
  const unsigned long long nraw = 4ull * st->swords;
  const unsigned long long nch = (nraw + kLzChunk - 1) / kLzChunk;
  const unsigned long long per = (nch + nt - 1) / nt;
  const unsigned long long lo = min(nch, tid * per), hi = min(nch, lo + per);
  unsigned long long sum = 0;
  for (unsigned long long i = lo; i < hi; ++i) sum += sizes[i] & 0x7FFFFFFFu;
  unsigned long long tot;
  unsigned long long pre = cta_exscan<unsigned long long>(sum, s_w, tot);
  const unsigned long long head = al16(16 + 4 * nch);
  for (unsigned long long i = lo; i < hi; ++i) {
    offs[i] = head + pre;
    pre += sizes[i] & 0x7FFFFFFFu;
  }
  const unsigned long long lzb = head + tot;
  const unsigned long long total = al16(off_st + lzb);
  if (total > cap) {
    if (tid == 0) st->err = PC_ERR_CAPACITY;
    return;
  }
  uint8_t* sec = out + off_st;
  for (unsigned long long i = tid; i < nch; i += nt) st_u32(sec + 16 + 4 * i, sizes[i]);
  for (unsigned long long i = 16 + 4 * nch + tid; i < head; i += nt) sec[i] = 0;
  for (unsigned long long i = off_st + lzb + tid; i < total; i += nt) out[i] = 0;
  if (tid == 0) {
    st_u32(sec, (unsigned int)nch);
    st_u32(sec + 4, (unsigned int)kLzChunk);
    st_u64(sec + 8, nraw);
    st->total = total;
    st->out_size = total;
  }
  if (tid < 256) {
    unsigned int cr = (unsigned int)tid;
    for (int k = 0; k < 8; ++k) cr = (cr >> 1) ^ (0xEDB88320u & (0u - (cr & 1u)));
    s_crc[tid] = cr;
  }
  __syncthreads();
  if (tid == 0) {
    st_u64(out + 216, total);
    st_u32(out + 228, *reinterpret_cast<const unsigned int*>(out + 228) | kFlagLossless);
    st_u64(out + 240, lzb);
    unsigned int crc = 0xFFFFFFFFu;
    for (int i = 0; i < 252; ++i) crc = s_crc[(crc ^ out[i]) & 0xFFu] ^ (crc >> 8);
    st_u32(out + 252, crc ^ 0xFFFFFFFFu);
  }
}

// One CTA per chunk: its slot (tokens or the raw chunk) into the section.
__global__ void __launch_bounds__(256) k_lz_gather(const uint8_t* __restrict__ slots,
                                                   const unsigned int* __restrict__ sizes,
                                                   const unsigned long long* __restrict__ offs, const State* st,
                                                   uint8_t* out) {
  if (st->err) return;
  const unsigned long long c = blockIdx.x;
  if (c * kLzChunk >= 4ull * st->swords) return;
  const unsigned int n = sizes[c] & 0x7FFFFFFFu;
  const uint8_t* src = slots + c * kLzSlot;
  uint8_t* dst = out + st->off_st + offs[c];
  for (unsigned int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Decoding: the chunks' section offsets (one CTA; a damaged section header
// or table sets PC_ERR_CORRUPT), then one thread per chunk into the raw
// stream buffer (token bounds and distances checked).
__global__ void __launch_bounds__(1024) k_lz_offsets(const uint8_t* __restrict__ sec, unsigned long long lzb,
                                                     unsigned long long nraw, unsigned long long* offs, int* err) {
  __shared__ unsigned long long s_w[32];
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const unsigned long long nch = (nraw + kLzChunk - 1) / kLzChunk;
  if (tid == 0) {
    bool bad = lzb < 16;
    if (!bad)
      bad = *reinterpret_cast<const unsigned int*>(sec) != nch ||
            *reinterpret_cast<const unsigned int*>(sec + 4) != (unsigned int)kLzChunk ||
            *reinterpret_cast<const unsigned long long*>(sec + 8) != nraw || al16(16 + 4 * nch) > lzb;
    s_bad = bad;
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) atomicExch(err, PC_ERR_CORRUPT);
    return;
  }
  const unsigned int* tab = reinterpret_cast<const unsigned int*>(sec + 16);
  const unsigned long long per = (nch + nt - 1) / nt;
  const unsigned long long lo = min(nch, tid * per), hi = min(nch, lo + per);
  unsigned long long sum = 0;
  for (unsigned long long i = lo; i < hi; ++i) sum += tab[i] & 0x7FFFFFFFu;
  unsigned long long tot;
  unsigned long long pre = cta_exscan<unsigned long long>(sum, s_w, tot);
  const unsigned long long head = al16(16 + 4 * nch);
  for (unsigned long long i = lo; i < hi; ++i) {
    offs[i] = head + pre;
    pre += tab[i] & 0x7FFFFFFFu;
  }
  if (tid == 0 && head + tot != lzb) atomicExch(err, PC_ERR_CORRUPT);
}

// One warp per chunk: lane 0 reads each control byte; the lanes copy literal
// runs, and matches in steps no longer than the distance (every source byte
// is written before it is read).
__global__ void __launch_bounds__(32 * kLzWarps) k_lz_decode(const uint8_t* __restrict__ sec, unsigned long long nraw,
                                                             const unsigned long long* __restrict__ offs, uint8_t* raw,
                                                             int* err) {
  const unsigned long long nch = (nraw + kLzChunk - 1) / kLzChunk;
  const int lane = threadIdx.x & 31;
  const unsigned long long c = (unsigned long long)blockIdx.x * kLzWarps + (threadIdx.x >> 5);
  if (c >= nch || *reinterpret_cast<volatile int*>(err)) return;
  const unsigned int e = reinterpret_cast<const unsigned int*>(sec + 16)[c];
  const unsigned long long sz = e & 0x7FFFFFFFu;
  const unsigned long long n = nraw - c * kLzChunk < (unsigned long long)kLzChunk ? nraw - c * kLzChunk : kLzChunk;
  const uint8_t* t = sec + offs[c];
  uint8_t* d = raw + c * kLzChunk;
  bool bad = false;
  if (e >> 31) {
    if (sz != n) bad = true;
    else
      for (unsigned long long i = lane; i < n; i += 32) d[i] = t[i];
  } else {
    unsigned long long p = 0, q = 0;
    while (p < sz) {
      const unsigned int cb = t[p++];
      if (cb < 128u) {
        const unsigned long long L = cb + 1;
        if (p + L > sz || q + L > n) { bad = true; break; }
        for (unsigned long long k = lane; k < L; k += 32) d[q + k] = t[p + k];
        p += L;
        q += L;
      } else {
        const unsigned long long L = cb - 128u + 4u;
        if (p + 2 > sz) { bad = true; break; }
        const unsigned long long dist = (unsigned long long)t[p] | ((unsigned long long)t[p + 1] << 8);
        p += 2;
        if (dist < 1 || dist > q || q + L > n) { bad = true; break; }
        const unsigned long long stp = dist < 32 ? dist : 32;
        for (unsigned long long k0 = 0; k0 < L; k0 += stp) {
          if (lane < stp && k0 + lane < L) d[q + k0 + lane] = d[q + k0 + lane - dist];
          __syncwarp();
        }
        q += L;
      }
      __syncwarp();
    }
    if (q != n) bad = true;
  }
  if (bad && lane == 0) atomicExch(err, PC_ERR_CORRUPT);
}

unsigned long long lz_chunks_max(unsigned long long raw_max) { return (raw_max + kLzChunk - 1) / kLzChunk; }

int launch_lz_encode(uint8_t* out, unsigned long long cap, State* st, const LzBufs& lb, cudaStream_t s) {
  ProfScope p(kStPack, s);
  const unsigned long long nch = lb.nch_max;
  if (nch == 0) return PC_OK;
  const size_t sm = (size_t)kLzWarps * (kLzChunk + 2 * (1 << kLzHashBits));
  if (cudaFuncSetAttribute(k_lz_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return PC_ERR_CUDA;
  k_lz_encode<<<(unsigned int)((nch + kLzWarps - 1) / kLzWarps), 32 * kLzWarps, sm, s>>>(out, nch, lb.slots, lb.sizes,
                                                                                         st);
  k_lz_layout<<<1, 1024, 0, s>>>(lb.sizes, lb.offs, st, out, cap);
  k_lz_gather<<<(unsigned int)nch, 256, 0, s>>>(lb.slots, lb.sizes, lb.offs, st, out);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

int launch_lz_decode(const uint8_t* sec, unsigned long long lzb, unsigned long long nraw, uint8_t* raw,
                     unsigned long long* offs, int* err, cudaStream_t s) {
  const unsigned long long nch = (nraw + kLzChunk - 1) / kLzChunk;
  if (nch == 0) return PC_OK;
  ProfScope p(kStDecScan, s);
  k_lz_offsets<<<1, 1024, 0, s>>>(sec, lzb, nraw, offs, err);
  k_lz_decode<<<(unsigned int)((nch + kLzWarps - 1) / kLzWarps), 32 * kLzWarps, 0, s>>>(sec, nraw, offs, raw, err);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // namespace pc
