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
// a length exceeds 24.  Code words are assigned along the symbol list ordered
// most frequent first (the sorted leaves reversed), where lengths never
// decrease: consecutive codes per length, as in RFC 1951 Section 3.2.2 and
// ITU-T T.81 Annex C.  Leaves are sorted by a stable radix sort on counts.
#include "pc_kernels.cuh"
#include "pc_profile.cuh"

namespace pc {

constexpr int kCbThreads = 1024;
constexpr int kCbSmemN = 12288;  // merge rounds run in shared memory once the list is this short
constexpr size_t kCbSmem = (size_t)kCbSmemN * 16;  // two lists of packed (weight, id) nodes

// Stable LSD radix sort (8-bit digits) of (key, val) pairs by key, one CTA of
// 32 warps.  Each warp owns a contiguous tile; per-warp digit counts give
// every (warp, digit) its output offset; inside a warp equal digits are
// ranked in lane order with __match_any_sync, so the sort is stable.
__device__ void cta_radix_sort(unsigned int* k0, uint16_t* v0, unsigned int* k1, uint16_t* v1, int n, int npass,
                               unsigned int* s_hist /* [32][256] */, unsigned int* s_tot /* [256] */,
                               unsigned long long* s_scan, unsigned int*& kout, uint16_t*& vout) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int T = (n + 31) / 32;
  const int lo = min(n, wid * T), hi = min(n, lo + T);
  unsigned int* ki = k0;
  uint16_t* vi = v0;
  unsigned int* ko = k1;
  uint16_t* vo = v1;
  for (int pass = 0; pass < npass; ++pass) {
    const int sh = 8 * pass;
    for (int i = tid; i < 32 * 256; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    for (int i = lo + lane; i < hi; i += 32) atomicAdd(&s_hist[wid * 256 + ((ki[i] >> sh) & 255u)], 1u);
    __syncthreads();
    unsigned long long col = 0;
    if (tid < 256)
      for (int w = 0; w < 32; ++w) col += s_hist[w * 256 + tid];
    unsigned long long tot;
    const unsigned long long base = cta_exscan<unsigned long long>(tid < 256 ? col : 0ull, s_scan, tot);
    if (tid < 256) {
      unsigned int run = (unsigned int)base;
      for (int w = 0; w < 32; ++w) {
        const unsigned int c = s_hist[w * 256 + tid];
        s_hist[w * 256 + tid] = run;
        run += c;
      }
    }
    __syncthreads();
    for (int c0 = lo; c0 < hi; c0 += 32) {
      const int i = c0 + lane;
      const bool valid = i < hi;
      const unsigned int key = valid ? ki[i] : 0u;
      const unsigned int d = valid ? ((key >> sh) & 255u) : 256u + (unsigned int)lane;
      const unsigned int peers = __match_any_sync(0xFFFFFFFFu, d);
      const unsigned int rank = __popc(peers & ((1u << lane) - 1u));
      if (valid) {
        const unsigned int pos = s_hist[wid * 256 + d] + rank;
        ko[pos] = key;
        vo[pos] = vi[i];
      }
      __syncwarp();
      if (valid && lane == 31 - __clz(peers)) s_hist[wid * 256 + d] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    unsigned int* tk = ki; ki = ko; ko = tk;
    uint16_t* tv = vi; vi = vo; vo = tv;
  }
  kout = ki;
  vout = vi;
  (void)s_tot;
}

// One merge round on a sorted list of packed nodes (weight << 32 | id),
// leaves first in (weight, symbol) order.  Joins every pair (L2i, L2i+1)
// whose second element weighs at most t1 = w(L0) + w(L1) (all of them precede
// t1 in the total order), records the new nodes' parents, and merges the new
// nodes (already sorted) with the rest of the list into `out`: an old node
// goes first on equal weight.  Each thread finds where its share of the
// output starts by a co-rank search, then merges sequentially.
__device__ __forceinline__ unsigned long long nn_node(const unsigned long long* in, int i, int next) {
  const unsigned long long a = in[2 * i], b = in[2 * i + 1];
  return (((a >> 32) + (b >> 32)) << 32) | (unsigned long long)(next + i);
}

__device__ int huff_round(const unsigned long long* in, unsigned long long* out, int len, int next,
                          unsigned int* parent, unsigned long long* s_scan, int& njoin) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const unsigned long long t1 = (in[0] >> 32) + (in[1] >> 32);
  int c = 0;
  for (int i = tid; i < len / 2; i += nt) c += (in[2 * i + 1] >> 32) <= t1;
  unsigned long long jt;
  cta_exscan<unsigned long long>((unsigned long long)c, s_scan, jt);
  const int j = (int)jt;
  for (int i = tid; i < j; i += nt) {
    parent[(unsigned int)in[2 * i]] = (unsigned int)(next + i);
    parent[(unsigned int)in[2 * i + 1]] = (unsigned int)(next + i);
  }
  const unsigned long long* R = in + 2 * j;
  const int lenR = len - 2 * j;
  const int total = lenR + j;
  const int per = (total + nt - 1) / nt;
  const int k0 = min(total, tid * per), k1 = min(total, k0 + per);
  if (k0 < k1) {
    // co-rank: a elements of R and b = k0 - a of N precede output position k0
    int lo = max(0, k0 - j), hi = min(k0, lenR);
    while (lo < hi) {
      const int a = (lo + hi) >> 1;  // try taking a elements of R
      const int b = k0 - a;
      // R[a] must come after N[b-1]: w(N[b-1]) < w(R[a]) (ties put R first)
      if (b > 0 && a < lenR && (nn_node(in, b - 1, next) >> 32) >= (R[a] >> 32)) lo = a + 1;
      else hi = a;
    }
    int a = lo, b = k0 - lo;
    for (int k = k0; k < k1; ++k) {
      const bool takeR = b >= j || (a < lenR && (R[a] >> 32) <= (nn_node(in, b, next) >> 32));
      out[k] = takeR ? R[a] : nn_node(in, b, next);
      if (takeR) ++a; else ++b;
    }
  }
  __syncthreads();
  njoin = j;
  return total;
}

// Depth of every leaf from the parent links; counts per depth into s_bits.
__device__ void huff_depths(const unsigned int* parent, unsigned short* depth, const int* rstart, int n, int rounds,
                            int* s_bits) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int next = 2 * n - 1, root = next - 1;
  if (tid == 0) depth[root] = 0;
  __syncthreads();
  for (int r = rounds - 1; r >= 0; --r) {
    const int a = rstart[r], b = (r + 1 < rounds) ? rstart[r + 1] : next;
    for (int id = a + tid; id < b; id += nt)
      if (id != root) depth[id] = (unsigned short)(depth[parent[id]] + 1);
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) {
    const int d = (int)depth[parent[i]] + 1;
    atomicAdd(&s_bits[d < 127 ? d : 127], 1);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kCbThreads) k_codebook(const unsigned long long* __restrict__ hist, int m,
                                                         uint8_t* lens, uint32_t* cw, State* st, HuffScratch hs,
                                                         uint8_t* out, unsigned long long nblocks,
                                                         unsigned long long off_cb, unsigned long long cap) {
  extern __shared__ __align__(16) unsigned char arena[];
  __shared__ unsigned long long s_scan[32];
  __shared__ int s_bits[128];
  __shared__ unsigned int s_first[32], s_offs[32], s_lend[32], s_tot[256];
  __shared__ int s_u[4];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nsym = 1 << m;
  if (st->err) return;
  // Only entries of used symbols are ever read, so the length and code
  // tables are not cleared.  Compaction: used symbols in symbol order, with
  // their counts; each warp reads a contiguous range, 8 loads in flight.
  const int lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  const int per = (nsym + nwarp - 1) / nwarp;
  const int lo = min(nsym, wid * per), hi = min(nsym, lo + per);
  constexpr int U = 8;
  unsigned long long cnt = 0, mx = 0;
  for (int s0 = lo; s0 < hi; s0 += 32 * U) {
    unsigned long long h[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + 32 * u + lane;
      h[u] = s < hi ? hist[s] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      mx = max(mx, h[u]);
      cnt += __popc(__ballot_sync(0xFFFFFFFFu, h[u] > 0));
    }
  }
  unsigned long long tot;
  const unsigned long long pre = cta_exscan<unsigned long long>(lane == 0 ? cnt : 0ull, s_scan, tot);
  const int n = (int)tot;
  unsigned int* k0 = reinterpret_cast<unsigned int*>(hs.key);
  unsigned int* k1 = k0 + nsym;
  uint16_t* v0 = reinterpret_cast<uint16_t*>(hs.symord);
  uint16_t* v1 = v0 + nsym;
  {
    int p = (int)__shfl_sync(0xFFFFFFFFu, pre, 0);
    for (int s0 = lo; s0 < hi; s0 += 32 * U) {
      unsigned long long h[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int s = s0 + 32 * u + lane;
        h[u] = s < hi ? hist[s] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned int bal = __ballot_sync(0xFFFFFFFFu, h[u] > 0);
        if (h[u] > 0) {
          const int q = p + __popc(bal & ((1u << lane) - 1u));
          k0[q] = (unsigned int)h[u];
          v0[q] = (uint16_t)(s0 + 32 * u + lane);
        }
        p += __popc(bal);
      }
    }
  }
  // largest count -> number of radix passes
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  if ((tid & 31) == 0) s_scan[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    unsigned long long m2 = 0;
    for (int i = 0; i < 32; ++i) m2 = max(m2, s_scan[i]);
    int np = 0;
    while (np < 4 && (m2 >> (8 * np)) != 0) ++np;
    s_u[1] = np;
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
      const unsigned int s = v0[0];
      lens[s] = 1;
      cw[s] = 1u << 24;
      st_u32(out + off_cb, s | (1u << 16));
    }
    for (unsigned long long i = off_cb + 4ull * n + tid; i < off_bb; i += nt) out[i] = 0;
    return;
  }
  // leaves sorted by (count, symbol): stable sort by count of the symbol-ordered list
  unsigned int* ks;
  uint16_t* vs;
  cta_radix_sort(k0, v0, k1, v1, n, s_u[1], reinterpret_cast<unsigned int*>(arena), s_tot, s_scan, ks, vs);
  for (int i = tid; i < 128; i += nt) s_bits[i] = 0;
  // merge rounds: in the workspace while the list is long, in shared memory after
  unsigned long long* ga = reinterpret_cast<unsigned long long*>(hs.w);
  unsigned long long* gb = ga + nsym;
  unsigned long long* sa = reinterpret_cast<unsigned long long*>(arena);
  unsigned long long* sb = sa + kCbSmemN;
  unsigned int* parent = reinterpret_cast<unsigned int*>(hs.parent);
  const bool start_smem = n <= kCbSmemN;
  unsigned long long* la = start_smem ? sa : ga;
  unsigned long long* lb = start_smem ? sb : gb;
  for (int i = tid; i < n; i += nt) la[i] = ((unsigned long long)ks[i] << 32) | (unsigned long long)i;
  __syncthreads();
  int len = n, next = n, rounds = 0;
  bool in_smem = start_smem;
  while (len > 1) {
    if (tid == 0) hs.rstart[rounds] = next;
    int j;
    len = huff_round(la, lb, len, next, parent, s_scan, j);
    next += j;
    ++rounds;
    if (!in_smem && len <= kCbSmemN) {
      for (int i = tid; i < len; i += nt) sa[i] = lb[i];
      __syncthreads();
      la = sa;
      lb = sb;
      in_smem = true;
    } else {
      unsigned long long* t = la; la = lb; lb = t;
    }
  }
  __syncthreads();
  const int nnode = 2 * n - 1;
  if ((size_t)nnode * 6 <= kCbSmem) {
    // walk the tree in shared memory: parent links copied in, depths beside them
    unsigned int* sp = reinterpret_cast<unsigned int*>(arena);
    unsigned short* sd = reinterpret_cast<unsigned short*>(sp + nnode);
    for (int i = tid; i < nnode - 1; i += nt) sp[i] = parent[i];
    __syncthreads();
    huff_depths(sp, sd, hs.rstart, n, rounds, s_bits);
  } else {
    huff_depths(parent, reinterpret_cast<unsigned short*>(hs.depth), hs.rstart, n, rounds, s_bits);
  }
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
    // leaves (ascending count) take lengths from the longest down: leaf ranks
    // below s_lend[l] have length >= l
    unsigned int cum = 0;
    for (int l = 31; l >= 1; --l) {
      if (l <= maxlen) cum += (unsigned int)s_bits[l];
      s_lend[l] = cum;
    }
    s_lend[0] = cum;
    unsigned int code = 0, off = 0;
    for (int l = 1; l <= kLmax; ++l) {
      const unsigned int prevc = l > 1 ? (unsigned int)s_bits[l - 1] : 0u;
      code = (code + prevc) << 1;
      off += prevc;
      s_first[l] = code;
      s_offs[l] = off;
    }
  }
  __syncthreads();
  const int maxlen = s_u[0];
  // canonical order: most frequent first (the sorted leaf list reversed)
  for (int i = tid; i < n; i += nt) {
    const unsigned int leaf = (unsigned int)(n - 1 - i);
    // length = largest l with leaf < s_lend[l] (s_lend decreases with l)
    int lo2 = 1, hi2 = maxlen;
    while (lo2 < hi2) {
      const int mid = (lo2 + hi2 + 1) >> 1;
      if (leaf < s_lend[mid]) lo2 = mid; else hi2 = mid - 1;
    }
    const int l = lo2;
    const unsigned int sym = vs[leaf];
    lens[sym] = (uint8_t)l;
    cw[sym] = (s_first[l] + ((unsigned int)i - s_offs[l])) | ((unsigned int)l << 24);
    st_u32(out + off_cb + 4ull * i, sym | ((unsigned int)l << 16));
  }
  for (unsigned long long i = off_cb + 4ull * n + tid; i < off_bb; i += nt) out[i] = 0;
}

int launch_codebook(const unsigned long long* hist, int m, uint8_t* lens, uint32_t* cw, State* st,
                    const HuffScratch& hs, uint8_t* out, const Geo& g, const HdrInfo& hi, cudaStream_t s) {
  const size_t smem = kCbSmem;
  if (cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PC_ERR_CUDA;
  ProfScope p(kStCodebook, s);
  k_codebook<<<1, kCbThreads, smem, s>>>(hist, m, lens, cw, st, hs, out, (unsigned long long)g.nblocks, hi.off_cb,
                                         hi.cap);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // namespace pc
