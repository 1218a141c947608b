// a10: Huffman code lengths and canonical code words, one CTA.
//
// Huffman's rule (repeatedly join the two lightest nodes) under the total
// order (weight, leaf before internal node, leaves by symbol, internal nodes
// by creation) is evaluated in parallel rounds.  With the available nodes in
// one sorted list L, joining L0+L1 makes t1; the sequential algorithm then
// joins the pairs (L2,L3), (L4,L5), ... for as long as the second element of
// the pair weighs at most t1, because every such element precedes t1 (and all
// nodes made after it) in the order.  A round therefore creates all those
// nodes at once and merges them (they come out already sorted) back into the
// rest of the list; the result is the sequential algorithm's tree exactly.
// Lengths are then handed out by rank from the per-length counts (the lightest
// leaf gets the longest length), with the ITU-T T.81 Annex K.3 adjustment when
// a length exceeds 24, and canonical code words follow RFC 1951 Section 3.2.2.
#include "pc_kernels.cuh"

namespace pc {

constexpr int kCbThreads = 1024;
constexpr int kCbSmemN = 4096;  // node arrays live in shared memory up to this many leaves

__device__ void cta_bitonic(unsigned long long* a, int np) {
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long x = a[i], y = a[ixj];
          const bool up = (i & k) == 0;
          if ((x > y) == up) { a[i] = y; a[ixj] = x; }
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kCbThreads) k_codebook(const unsigned long long* __restrict__ hist, int m,
                                                         uint8_t* lens, uint32_t* cw, State* st, HuffScratch hs,
                                                         uint8_t* out, unsigned long long nblocks,
                                                         unsigned long long off_cb, unsigned long long cap) {
  extern __shared__ __align__(16) unsigned char arena[];
  __shared__ unsigned long long s_scan[32];
  __shared__ int s_bits[128];
  __shared__ unsigned int s_first[32], s_offs[32], s_lstart[32];
  __shared__ int s_u[4];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nsym = 1 << m;
  if (st->err) return;
  for (int i = tid; i < nsym; i += nt) { lens[i] = 0; cw[i] = 0; }
  // compaction: used symbols in symbol order
  const int per = (nsym + nt - 1) / nt;
  const int lo = min(nsym, tid * per), hi = min(nsym, lo + per);
  unsigned long long cnt = 0;
  for (int s = lo; s < hi; ++s) cnt += hist[s] > 0;
  unsigned long long tot;
  unsigned long long pre = cta_exscan<unsigned long long>(cnt, s_scan, tot);
  const int n = (int)tot;
  // node arrays: shared memory for small alphabets, workspace otherwise
  const bool small = n <= kCbSmemN;
  unsigned long long* key = small ? reinterpret_cast<unsigned long long*>(arena) : hs.key;
  unsigned long long* w = small ? key + kCbSmemN : hs.w;
  int* parent = small ? reinterpret_cast<int*>(w + 2 * kCbSmemN) : hs.parent;
  int* la = small ? parent + 2 * kCbSmemN : hs.la;
  int* lb = small ? la + kCbSmemN : hs.lb;
  int* depth = la;  // reuses la/lb (2n ints) once the rounds are done
  int* rstart = hs.rstart;
  {
    int p = (int)pre;
    for (int s = lo; s < hi; ++s) {
      const unsigned long long h = hist[s];
      if (h > 0) {
        hs.symord[p] = (unsigned int)s;
        key[p] = (h << 16) | (unsigned long long)s;
        ++p;
      }
    }
  }
  const unsigned long long off_bb = al16(off_cb + 4ull * (unsigned long long)n);
  const unsigned long long off_bn = al16(off_bb + 4ull * nblocks);
  if (tid == 0) {
    st->n_used = (unsigned int)n;
    st->off_cb = off_cb;
    st->off_bb = off_bb;
    st->off_bn = off_bn;
    if (off_bn + 2ull * nblocks > cap) st->err = PC_ERR_CAPACITY;
  }
  __syncthreads();
  if (st->err) return;
  if (n <= 1) {
    if (n == 1 && tid == 0) {
      const unsigned int s = hs.symord[0];
      lens[s] = 1;
      cw[s] = 0;
      st_u32(out + off_cb, s | (1u << 16));
    }
    for (unsigned long long i = off_cb + 4ull * n + tid; i < off_bb; i += nt) out[i] = 0;
    return;
  }
  int np = 1;
  while (np < n) np <<= 1;
  for (int i = n + tid; i < np; i += nt) key[i] = ~0ull;
  __syncthreads();
  cta_bitonic(key, np);
  // leaves: sorted by (freq, symbol)
  for (int i = tid; i < n; i += nt) { w[i] = key[i] >> 16; la[i] = i; }
  __syncthreads();
  int len = n, next = n, round = 0;
  while (len > 1) {
    const unsigned long long t1 = w[la[0]] + w[la[1]];
    int c = 0;
    for (int i = tid; i < len / 2; i += nt) c += w[la[2 * i + 1]] <= t1;
    unsigned long long jt;
    cta_exscan<unsigned long long>((unsigned long long)c, s_scan, jt);
    const int j = (int)jt;
    for (int i = tid; i < j; i += nt) {
      const int a = la[2 * i], b = la[2 * i + 1];
      w[next + i] = w[a] + w[b];
      parent[a] = next + i;
      parent[b] = next + i;
    }
    if (tid == 0) rstart[round] = next;
    __syncthreads();
    const int lenR = len - 2 * j;
    for (int a = tid; a < lenR; a += nt) {
      const int id = la[2 * j + a];
      const unsigned long long wa = w[id];
      int l0 = 0, h0 = j;
      while (l0 < h0) {
        const int mid = (l0 + h0) >> 1;
        if (w[next + mid] < wa) l0 = mid + 1; else h0 = mid;
      }
      lb[a + l0] = id;
    }
    for (int bi = tid; bi < j; bi += nt) {
      const unsigned long long wb = w[next + bi];
      int l0 = 0, h0 = lenR;
      while (l0 < h0) {
        const int mid = (l0 + h0) >> 1;
        if (w[la[2 * j + mid]] <= wb) l0 = mid + 1; else h0 = mid;
      }
      lb[bi + l0] = next + bi;
    }
    __syncthreads();
    int* tmp = la; la = lb; lb = tmp;
    len = lenR + j;
    next += j;
    ++round;
  }
  // depth: the root is the single node of the last round; parents come later
  const int root = next - 1;
  depth = small ? parent + 2 * kCbSmemN : hs.depth;  // shared: the la/lb region, 2 * kCbSmemN ints
  if (tid == 0) depth[root] = 0;
  for (int i = tid; i < 128; i += nt) s_bits[i] = 0;
  __syncthreads();
  for (int r = round - 1; r >= 0; --r) {
    const int a = rstart[r], b = (r + 1 < round) ? rstart[r + 1] : next;
    for (int id = a + tid; id < b; id += nt)
      if (id != root) depth[id] = depth[parent[id]] + 1;
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) {
    const int d = depth[parent[i]] + 1;
    atomicAdd(&s_bits[d < 127 ? d : 127], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int maxlen = 0;
    for (int l = 1; l < 128; ++l)
      if (s_bits[l]) maxlen = l;
    if (maxlen > kLmax) {
      for (int i = maxlen; i > kLmax; --i) {
        while (s_bits[i] > 0) {
          int jj = i - 2;
          while (jj > 0 && s_bits[jj] == 0) --jj;
          s_bits[i] -= 2;
          s_bits[i - 1] += 1;
          s_bits[jj + 1] += 2;
          s_bits[jj] -= 1;
        }
      }
      maxlen = kLmax;
    }
    s_u[0] = maxlen;
    unsigned int cum = 0;
    for (int l = maxlen; l >= 1; --l) { s_lstart[l] = cum; cum += (unsigned int)s_bits[l]; }
    unsigned int code = 0, off = 0;
    s_first[0] = 0;
    s_offs[0] = 0;
    for (int l = 1; l <= kLmax; ++l) {
      code = (code + (unsigned int)(l > 1 ? s_bits[l - 1] : 0)) << 1;
      s_first[l] = code;
      off += (unsigned int)(l > 1 ? s_bits[l - 1] : 0);
      s_offs[l] = off;
    }
  }
  __syncthreads();
  const int maxlen = s_u[0];
  // lengths by rank; second sort key (length, symbol) goes into w
  unsigned long long* key2 = w;
  for (int i = tid; i < np; i += nt) {
    if (i < n) {
      int l = maxlen;
      while (l > 1 && !((unsigned int)i >= s_lstart[l] && (unsigned int)i < s_lstart[l] + (unsigned int)s_bits[l])) --l;
      const unsigned int sym = (unsigned int)(key[i] & 0xFFFFull);
      lens[sym] = (uint8_t)l;
      key2[i] = ((unsigned long long)l << 16) | sym;
    } else {
      key2[i] = ~0ull;
    }
  }
  __syncthreads();
  cta_bitonic(key2, np);
  for (int p = tid; p < n; p += nt) {
    const unsigned int l = (unsigned int)(key2[p] >> 16), sym = (unsigned int)(key2[p] & 0xFFFFull);
    cw[sym] = s_first[l] + ((unsigned int)p - s_offs[l]);
  }
  __syncthreads();
  for (int p = tid; p < n; p += nt) {
    const unsigned int sym = hs.symord[p];
    st_u32(out + off_cb + 4ull * p, sym | ((unsigned int)lens[sym] << 16));
  }
  for (unsigned long long i = off_cb + 4ull * n + tid; i < off_bb; i += nt) out[i] = 0;
}

int launch_codebook(const unsigned long long* hist, int m, uint8_t* lens, uint32_t* cw, State* st,
                    const HuffScratch& hs, uint8_t* out, const Geo& g, const HdrInfo& hi, cudaStream_t s) {
  const size_t smem = (size_t)kCbSmemN * 8 * 3 + (size_t)kCbSmemN * 4 * 4;  // key, w (2x), parent (2x), la, lb
  if (cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PC_ERR_CUDA;
  k_codebook<<<1, kCbThreads, smem, s>>>(hist, m, lens, cw, st, hs, out, (unsigned long long)g.nblocks, hi.off_cb,
                                         hi.cap);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // namespace pc
