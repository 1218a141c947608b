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
//
// Node weights are held in 32 bits: the field has fewer than 2^32 points,
// which the entry points check.  Everything that fits runs in shared memory;
// for many used symbols the sort and the first (long) merge rounds run in
// the workspace, staged through shared memory in tiles.
#include "pc_kernels.cuh"
#include "pc_profile.cuh"

namespace pc {

constexpr int kCbThreads = 1024;
constexpr size_t kCbSmem = 196608;  // dynamic shared memory arena
constexpr int kCbListN = 12288;     // merge lists (two of packed u64 nodes) in shared memory up to this length
constexpr int kCbTile = 12288;      // long rounds: output tile staged through shared memory
constexpr int kCbSortN = 13568;     // radix sort in shared memory up to this many leaves (12 B each + 32 KB counts)
constexpr int kRadixU = 4;          // 32-key chunks a warp loads before it ranks them

// Smallest x in [lo, hi] with pred(x), for pred false then true over the
// range (pred(hi) is taken as true and never evaluated).  All lanes of the
// calling warp take part and return the same x; each step probes 32 points.
template <typename P>
__device__ __forceinline__ int warp_first_true(int lo, int hi, P pred) {
  const int lane = threadIdx.x & 31;
  while (lo < hi) {
    const int step = (hi - lo + 31) / 32;
    const int x = lo + (lane + 1) * step - 1;
    const bool t = x >= hi ? true : pred(x);
    const unsigned int b = __ballot_sync(0xFFFFFFFFu, t);
    if (b == 0u) return hi;
    const int f = __ffs(b) - 1;
    const int xf = lo + (f + 1) * step - 1;
    lo = lo + f * step;
    hi = min(hi, xf);
  }
  return lo;
}

// Stable LSD radix sort (8-bit digits) of (key, val) pairs by key, one CTA of
// 32 warps: input (kin, vin), result in (kout, vout), two temporaries for the
// passes in between.  Each warp owns a contiguous tile; per-warp digit counts
// give every (warp, digit) its output offset; inside a warp equal digits are
// ranked in lane order with __match_any_sync, so the sort is stable.
__device__ void cta_radix_sort(const unsigned int* kin, const uint16_t* vin, unsigned int* ka, uint16_t* va,
                               unsigned int* kb, uint16_t* vb, unsigned int* kout, uint16_t* vout, int n, int npass,
                               unsigned int* s_hist /* [32][256] */, unsigned long long* s_scan) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int T = (n + 31) / 32;
  const int lo = min(n, wid * T), hi = min(n, lo + T);
  const unsigned int* ki = kin;
  const uint16_t* vi = vin;
  for (int pass = 0; pass < npass; ++pass) {
    unsigned int* ko = pass == npass - 1 ? kout : ((pass & 1) ? kb : ka);
    uint16_t* vo = pass == npass - 1 ? vout : ((pass & 1) ? vb : va);
    const int sh = 8 * pass;
    for (int i = tid; i < 32 * 256; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    for (int c0 = lo; c0 < hi; c0 += 32 * kRadixU) {
      unsigned int key[kRadixU];
#pragma unroll
      for (int u = 0; u < kRadixU; ++u) {
        const int i = c0 + 32 * u + lane;
        key[u] = i < hi ? ki[i] : 0u;
      }
#pragma unroll
      for (int u = 0; u < kRadixU; ++u)
        if (c0 + 32 * u + lane < hi) atomicAdd(&s_hist[wid * 256 + ((key[u] >> sh) & 255u)], 1u);
    }
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
    for (int c0 = lo; c0 < hi; c0 += 32 * kRadixU) {
      unsigned int key[kRadixU];
      uint16_t val[kRadixU];
#pragma unroll
      for (int u = 0; u < kRadixU; ++u) {
        const int i = c0 + 32 * u + lane;
        key[u] = i < hi ? ki[i] : 0u;
        val[u] = i < hi ? vi[i] : (uint16_t)0;
      }
#pragma unroll
      for (int u = 0; u < kRadixU; ++u) {
        const bool valid = c0 + 32 * u + lane < hi;
        const unsigned int d = valid ? ((key[u] >> sh) & 255u) : 256u + (unsigned int)lane;
        const unsigned int peers = __match_any_sync(0xFFFFFFFFu, d);
        const unsigned int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid) {
          const unsigned int pos = s_hist[wid * 256 + d] + rank;
          ko[pos] = key[u];
          vo[pos] = val[u];
        }
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) s_hist[wid * 256 + d] += __popc(peers);
        __syncwarp();
      }
    }
    __syncthreads();
    ki = ko;
    vi = vo;
  }
}

// Merge rounds on a sorted list of packed nodes (weight << 32 | id), leaves
// first in (weight, symbol) order.  A round joins every pair (L2i, L2i+1)
// whose second element weighs at most t1 = w(L0) + w(L1) (all of them precede
// t1 in the total order; the list is sorted, so they are a prefix of the
// pairs), records the new nodes' parents, and merges the new nodes (already
// sorted) with the rest R of the list: an old node goes first on equal
// weight.  Output position k is reached after taking a nodes of R and k - a
// new ones, with a found by a co-rank search; each thread then merges its
// share sequentially.
__device__ __forceinline__ unsigned long long nn_node(const unsigned long long* in, int i, int next) {
  const unsigned long long a = in[2 * i], b = in[2 * i + 1];
  return (((a >> 32) + (b >> 32)) << 32) | (unsigned long long)(next + i);
}

__device__ __forceinline__ unsigned int wt(unsigned long long v) { return (unsigned int)(v >> 32); }

// Number of pairs joined in this round, found by warp 0 and shared.
__device__ __forceinline__ int round_joins(const unsigned long long* in, int len, int* s_j) {
  if (threadIdx.x < 32) {
    const unsigned long long t1 = (unsigned long long)wt(in[0]) + wt(in[1]);
    const int j = warp_first_true(0, len / 2, [&](int i) { return (unsigned long long)wt(in[2 * i + 1]) > t1; });
    if (threadIdx.x == 0) *s_j = j;
  }
  __syncthreads();
  return *s_j;
}

__device__ __forceinline__ void set_parents(const unsigned long long* in, int j, int next, unsigned int* parent) {
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    parent[(unsigned int)in[2 * i]] = (unsigned int)(next + i);
    parent[(unsigned int)in[2 * i + 1]] = (unsigned int)(next + i);
  }
}

// Merge of R[0, nR) and N[0, nN) (N given by the callable) into out[k0, k1)
// for this thread's share of [0, nR + nN); sequential from its co-rank.
template <typename NF>
__device__ __forceinline__ void merge_share(const unsigned long long* R, int nR, NF N, int nN, unsigned long long* out) {
  const int total = nR + nN;
  const int per = (total + (int)blockDim.x - 1) / (int)blockDim.x;
  const int k0 = min(total, (int)threadIdx.x * per), k1 = min(total, k0 + per);
  if (k0 >= k1) return;
  // smallest a such that N[k0-a-1] (if any) precedes R[a] (if any): w(N) < w(R)
  int lo = max(0, k0 - nN), hi = min(k0, nR);
  while (lo < hi) {
    const int a = (lo + hi) >> 1;
    const int b = k0 - a;
    if (b > 0 && a < nR && wt(N(b - 1)) >= wt(R[a])) lo = a + 1;
    else hi = a;
  }
  int a = lo, b = k0 - lo;
  for (int k = k0; k < k1; ++k) {
    const bool takeR = b >= nN || (a < nR && wt(R[a]) <= wt(N(b)));
    out[k] = takeR ? R[a] : N(b);
    if (takeR) ++a; else ++b;
  }
}

// One round with both lists in shared memory.
__device__ int huff_round_smem(const unsigned long long* in, unsigned long long* out, int len, int next,
                               unsigned int* parent, int* s_j, int& njoin) {
  const int j = round_joins(in, len, s_j);
  set_parents(in, j, next, parent);
  merge_share(in + 2 * j, len - 2 * j, [&](int b) { return nn_node(in, b, next); }, j, out);
  __syncthreads();
  njoin = j;
  return len - j;
}

// One round with the lists in the workspace: the output is cut into tiles of
// kCbTile; one warp per tile boundary finds its co-rank, then each tile's
// nodes are loaded into shared memory (coalesced) and merged there.
__device__ int huff_round_global(const unsigned long long* in, unsigned long long* out, int len, int next,
                                 unsigned int* parent, unsigned long long* sR, unsigned long long* sN, int* s_j,
                                 int* s_cr, int& njoin) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int j = round_joins(in, len, s_j);
  set_parents(in, j, next, parent);
  const unsigned long long* R = in + 2 * j;
  const int lenR = len - 2 * j;
  const int total = lenR + j;
  const int ntile = (total + kCbTile - 1) / kCbTile;  // <= 6 for 2^16 symbols
  if (wid <= ntile) {
    const int k = min(total, wid * kCbTile);
    const int a = warp_first_true(max(0, k - j), min(k, lenR), [&](int a) {
      const int b = k - a;
      return !(b > 0 && a < lenR && wt(nn_node(in, b - 1, next)) >= wt(R[a]));
    });
    if (lane == 0) s_cr[wid] = a;
  }
  __syncthreads();
  for (int t = 0; t < ntile; ++t) {
    const int k0 = t * kCbTile, k1 = min(total, k0 + kCbTile);
    const int a0 = s_cr[t], a1 = s_cr[t + 1];
    const int b0 = k0 - a0, b1 = k1 - a1;
    for (int i = tid; i < a1 - a0; i += nt) sR[i] = R[a0 + i];
    for (int i = tid; i < b1 - b0; i += nt) sN[i] = nn_node(in, b0 + i, next);
    __syncthreads();
    merge_share(sR, a1 - a0, [&](int b) { return sN[b]; }, b1 - b0, out + k0);
    __syncthreads();
  }
  njoin = j;
  return total;
}

// Depth of every leaf from the parent links, walked from the root down one
// round at a time; counts per depth into s_bits.
template <typename D>
__device__ void huff_depths(const unsigned int* parent, D* depth, const int* rstart, int n, int rounds, int* s_bits) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int next = 2 * n - 1, root = next - 1;
  if (tid == 0) depth[root] = 0;
  __syncthreads();
  for (int r = rounds - 1; r >= 0; --r) {
    const int a = rstart[r], b = (r + 1 < rounds) ? rstart[r + 1] : next;
    for (int id = a + tid; id < b; id += nt)
      if (id != root) depth[id] = (D)(depth[parent[id]] + 1);
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) {
    const int d = (int)depth[parent[i]] + 1;
    atomicAdd(&s_bits[d < 127 ? d : 127], 1);
  }
  __syncthreads();
}

// ITU-T T.81 Annex K.3 length limiting on the per-length counts, with the
// procedure's repeated single steps taken in batches.  Each step at level i
// moves a pair of leaves off level i (one to level i-1) and splits the
// deepest leaf at a level <= i-2 into two leaves one level down.  Splitting
// a leaf at level j and, depth first, every leaf that split creates down to
// level i-2 takes 2^(i-1-j) - 1 steps and leaves 2^(i-1-j) leaves at level
// i-1; whole such expansions are batched, a partial one descends a level.
__device__ void limit_lengths(int* bits, int maxlen, int lmax) {
  for (int i = maxlen; i > lmax; --i) {
    long long P = (bits[i] + 1) / 2;  // steps of the procedure at this level
    if (P <= 0) continue;
    bits[i] -= (int)(2 * P);
    bits[i - 1] += (int)P;
    const int D = i - 2;
    int j = D;
    while (j > 0 && bits[j] == 0) --j;
    while (P > 0) {
      if (j <= 0) {  // not reached for a valid tree; same step as the procedure's
        bits[0] -= 1;
        bits[1] += 2;
        --P;
        j = 1;
        continue;
      }
      const long long cost = (1ll << (D - j + 1)) - 1;
      const long long k = min((long long)bits[j], P / cost);
      bits[j] -= (int)k;
      bits[D + 1] += (int)(k << (D - j + 1));
      P -= k * cost;
      if (P == 0) break;
      if (bits[j] > 0) {  // P < cost: split one leaf; its children are now the deepest
        bits[j] -= 1;
        bits[j + 1] += 2;
        --P;
        ++j;
      } else {
        while (j > 0 && bits[j] == 0) --j;
      }
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
  __shared__ unsigned int s_first[32], s_offs[32], s_lend[32];
  __shared__ int s_u[4], s_cr[40];
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
  // workspace arrays (see the layout of HuffScratch): compacted input, two
  // sort temporaries, sorted output
  unsigned int* kc = reinterpret_cast<unsigned int*>(hs.key);
  uint16_t* vc = reinterpret_cast<uint16_t*>(hs.symord);
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
          kc[q] = (unsigned int)h[u];
          vc[q] = (uint16_t)(s0 + 32 * u + lane);
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
      const unsigned int s = vc[0];
      lens[s] = 1;
      cw[s] = 1u << 24;
      st_u32(out + off_cb, s | (1u << 16));
    }
    for (unsigned long long i = off_cb + 4ull * n + tid; i < off_bb; i += nt) out[i] = 0;
    return;
  }
  // leaves sorted by (count, symbol): stable sort by count of the symbol-ordered list
  unsigned int* ks = reinterpret_cast<unsigned int*>(hs.la);
  uint16_t* vs = reinterpret_cast<uint16_t*>(hs.lb);
  {
    unsigned int* s_hist = reinterpret_cast<unsigned int*>(arena);
    unsigned int *ka, *kb;
    uint16_t *va, *vb;
    if (n <= kCbSortN) {
      ka = s_hist + 32 * 256;
      kb = ka + kCbSortN;
      va = reinterpret_cast<uint16_t*>(kb + kCbSortN);
      vb = va + kCbSortN;
    } else {
      ka = kc + nsym;
      va = vc + nsym;
      kb = reinterpret_cast<unsigned int*>(hs.depth);
      vb = reinterpret_cast<uint16_t*>(kb + nsym);
    }
    cta_radix_sort(kc, vc, ka, va, kb, vb, ks, vs, n, s_u[1], s_hist, s_scan);
  }
  for (int i = tid; i < 128; i += nt) s_bits[i] = 0;
  // merge rounds: in the workspace while the list is long, in shared memory after
  unsigned long long* ga = reinterpret_cast<unsigned long long*>(hs.w);
  unsigned long long* gb = ga + nsym;
  unsigned long long* sa = reinterpret_cast<unsigned long long*>(arena);
  unsigned long long* sb = sa + kCbListN;
  unsigned int* parent = reinterpret_cast<unsigned int*>(hs.parent);
  bool in_smem = n <= kCbListN;
  unsigned long long* la = in_smem ? sa : ga;
  unsigned long long* lb = in_smem ? sb : gb;
  for (int i = tid; i < n; i += nt) la[i] = ((unsigned long long)ks[i] << 32) | (unsigned long long)i;
  __syncthreads();
  int len = n, next = n, rounds = 0;
  while (len > 1) {
    if (tid == 0) hs.rstart[rounds] = next;
    int j;
    if (in_smem) len = huff_round_smem(la, lb, len, next, parent, &s_u[2], j);
    else len = huff_round_global(la, lb, len, next, parent, sa, sb, &s_u[2], s_cr, j);
    next += j;
    ++rounds;
    if (!in_smem && len <= kCbListN) {
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
    // parent links from the workspace, depths (< 64 for 32-bit weights) in shared memory
    huff_depths(parent, reinterpret_cast<unsigned char*>(arena), hs.rstart, n, rounds, s_bits);
  }
  if (tid == 0) {
    int maxlen = 0;
    for (int l = 1; l < 128; ++l)
      if (s_bits[l]) maxlen = l;
    if (maxlen > kLmax) {
      limit_lengths(s_bits, maxlen, kLmax);
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
  constexpr int UA = 4;
  for (int i0 = 0; i0 < n; i0 += nt * UA) {
    unsigned int sym[UA];
#pragma unroll
    for (int u = 0; u < UA; ++u) {
      const int i = i0 + u * nt + tid;
      sym[u] = i < n ? vs[n - 1 - i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < UA; ++u) {
      const int i = i0 + u * nt + tid;
      if (i >= n) break;
      const unsigned int leaf = (unsigned int)(n - 1 - i);
      // length = largest l with leaf < s_lend[l] (s_lend decreases with l)
      int lo2 = 1, hi2 = maxlen;
      while (lo2 < hi2) {
        const int mid = (lo2 + hi2 + 1) >> 1;
        if (leaf < s_lend[mid]) lo2 = mid; else hi2 = mid - 1;
      }
      const int l = lo2;
      lens[sym[u]] = (uint8_t)l;
      cw[sym[u]] = (s_first[l] + ((unsigned int)i - s_offs[l])) | ((unsigned int)l << 24);
      st_u32(out + off_cb + 4ull * i, sym[u] | ((unsigned int)l << 16));
    }
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
