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
// ITU-T T.81 Annex C.  Leaves are sorted by count with a stable radix sort
// (in shared memory when they fit, else in the workspace).
//
// Node weights are held in 32 bits: the field has fewer than 2^32 points,
// which the entry points check.  Everything that fits runs in shared memory;
// for many used symbols the sort and the merge queues live in the workspace.
#include "pc_kernels.cuh"
#include "pc_profile.cuh"

namespace pc {

constexpr int kCbThreads = 1024;
constexpr size_t kCbSmem = 196608;  // dynamic shared memory arena
constexpr int kCbQueueN = 24576;    // merge queues (leaf and internal weights, u32) in shared memory up to this n

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

// Stable sort, by key, of (key, val) pairs held in shared memory: LSD radix
// with 4-bit digits, one counting pass per digit of the largest key.
//
// A counting pass: thread t owns the contiguous run [t E, t E + E) of the
// input and counts its digits (in 4-bit fields of one register, E < 16); the
// counts go to column t of a digit-major table, whose exclusive scan in
// (digit, thread) order gives each (digit, thread) its first output slot.
// The pass is stable without any ranking across threads.
constexpr int kSegN = 13568;  // pairs sorted in shared memory at once (E <= 14 with 1024 threads)

// One stable counting pass of ki/vi[0, n) into ko/vo by digit(key) in 0..15.
template <typename DF>
__device__ void count_pass(const unsigned int* ki, const uint16_t* vi, unsigned int* ko, uint16_t* vo, int n, DF digit,
                           unsigned short* s_cnt, unsigned long long* s_scan) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int E = (n + nt - 1) / nt;
  const int lo = min(n, t * E), hi = min(n, lo + E);
  unsigned long long c = 0;
  for (int i = lo; i < hi; ++i) c += 1ull << (4 * digit(ki[i]));
#pragma unroll
  for (int d = 0; d < 16; ++d) s_cnt[d * nt + t] = (unsigned short)((c >> (4 * d)) & 15u);
  __syncthreads();
  // this thread's 16 consecutive table entries, as two 16-byte words
  uint4* row = reinterpret_cast<uint4*>(s_cnt + 16 * t);
  uint4 w0 = row[0], w1 = row[1];
  unsigned int e[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
  unsigned int sum = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) sum += (e[u] & 0xFFFFu) + (e[u] >> 16);
  unsigned long long tot;
  unsigned int run = (unsigned int)cta_exscan<unsigned long long>(sum, s_scan, tot);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const unsigned int lo16 = run;
    run += e[u] & 0xFFFFu;
    const unsigned int hi16 = run;
    run += e[u] >> 16;
    e[u] = lo16 | (hi16 << 16);
  }
  row[0] = make_uint4(e[0], e[1], e[2], e[3]);
  row[1] = make_uint4(e[4], e[5], e[6], e[7]);
  __syncthreads();
  for (int i = lo; i < hi; ++i) {
    const unsigned int key = ki[i];
    const int d = digit(key);
    const unsigned int pos = s_cnt[d * nt + t];
    s_cnt[d * nt + t] = (unsigned short)(pos + 1u);
    ko[pos] = key;
    vo[pos] = vi[i];
  }
  __syncthreads();
}

// Sorts k0/v0[0, n) (k1/v1 is the other buffer) on npass 4-bit digits and
// writes the result to (kout, vout) in global memory.
__device__ void smem_sort(unsigned int* k0, uint16_t* v0, unsigned int* k1, uint16_t* v1, int n, int npass,
                          unsigned int* kout, uint16_t* vout, unsigned short* s_cnt, unsigned long long* s_scan) {
  int cur = 0;
#pragma unroll 1
  for (int pass = 0; pass < npass; ++pass) {
    const int sh = 4 * pass;
    auto dig = [=](unsigned int k) { return (int)((k >> sh) & 15u); };
    if (cur) count_pass(k1, v1, k0, v0, n, dig, s_cnt, s_scan);
    else count_pass(k0, v0, k1, v1, n, dig, s_cnt, s_scan);
    cur ^= 1;
  }
  const unsigned int* rk = cur ? k1 : k0;
  const uint16_t* rv = cur ? v1 : v0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    kout[i] = rk[i];
    vout[i] = rv[i];
  }
  __syncthreads();
}

constexpr int kRadixU8 = 4;  // 32-key chunks a warp loads before it ranks them

// Stable LSD radix sort (8-bit digits) of (key, val) pairs by key in global
// memory, one CTA of 32 warps: input (kin, vin), result in (kout, vout), two temporaries for the
// passes in between.  Each warp owns a contiguous tile; per-warp digit counts
// give every (warp, digit) its output offset; inside a warp equal digits are
// ranked in lane order with __match_any_sync, so the sort is stable.
__device__ void cta_radix_sort8(const unsigned int* kin, const uint16_t* vin, unsigned int* ka, uint16_t* va,
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
    for (int c0 = lo; c0 < hi; c0 += 32 * kRadixU8) {
      unsigned int key[kRadixU8];
#pragma unroll
      for (int u = 0; u < kRadixU8; ++u) {
        const int i = c0 + 32 * u + lane;
        key[u] = i < hi ? ki[i] : 0u;
      }
#pragma unroll
      for (int u = 0; u < kRadixU8; ++u)
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
    for (int c0 = lo; c0 < hi; c0 += 32 * kRadixU8) {
      unsigned int key[kRadixU8];
      uint16_t val[kRadixU8];
#pragma unroll
      for (int u = 0; u < kRadixU8; ++u) {
        const int i = c0 + 32 * u + lane;
        key[u] = i < hi ? ki[i] : 0u;
        val[u] = i < hi ? vi[i] : (uint16_t)0;
      }
#pragma unroll
      for (int u = 0; u < kRadixU8; ++u) {
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

// Merge rounds on two queues: the leaves A (weights sorted by (count,
// symbol), ids 0..n-1) and the internal nodes B (ids n, n+1, ... in order of
// creation).  Huffman's rule creates internal nodes in non-decreasing weight,
// so B stays sorted, and the available nodes in the total order are the merge
// of the unconsumed parts A[p..] and B[q..nb) with a leaf first on equal
// weight.  A round joins L0+L1 into t1 and, with it, every following pair
// (L2i, L2i+1) whose second element weighs at most t1: with c nodes of weight
// <= t1 available, that is j = c/2 pairs, made of the first 2j nodes of the
// merge (x of them leaves).  Only those 2j nodes are touched, so the rounds
// do O(n) work in all.  The weights fit 32 bits (fewer than 2^32 points).
struct TwoQ {
  int p, q, nb, j, x, cA, cB;
};

// Warp 0: the round's j and x from the queue heads; result in *s.
__device__ void two_queue_plan(const unsigned int* A, const unsigned int* B, int n, TwoQ* s) {
  if (threadIdx.x >= 32) return;
  const int p = s->p, q = s->q, nb = s->nb;
  // the first two nodes of the merge
  unsigned int w[2];
  int pa = p, qb = q;
  for (int r = 0; r < 2; ++r) {
    const bool leaf = pa < n && (qb >= nb || A[pa] <= B[qb]);
    w[r] = leaf ? A[pa] : B[qb];
    if (leaf) ++pa; else ++qb;
  }
  const unsigned int t1 = w[0] + w[1];
  const int cA = warp_first_true(p, n, [&](int i) { return A[i] > t1; }) - p;
  const int cB = warp_first_true(q, nb, [&](int i) { return B[i] > t1; }) - q;
  const int j = (cA + cB) / 2;
  const int k = 2 * j;
  // x leaves among the first k: B[y-1] must strictly precede A[x] (leaf first on ties)
  const int x = warp_first_true(max(0, k - cB), min(k, cA), [&](int xx) {
    const int y = k - xx;
    return !(y > 0 && xx < cA && B[q + y - 1] >= A[p + xx]);
  });
  if (threadIdx.x == 0) {
    s->j = j;
    s->x = x;
    s->cA = cA;
    s->cB = cB;
  }
}

// All threads: create this round's j nodes from the first 2j nodes of the
// merge of A[p, p+x) and B[q, q+2j-x); each thread takes a run of pairs,
// finds where it starts by a co-rank search and merges sequentially.
__device__ void two_queue_join(const unsigned int* A, unsigned int* B, int n, const TwoQ& s, unsigned int* parent,
                               int t, int nt) {
  const int j = s.j, x = s.x, y = 2 * j - s.x;
  const unsigned int* Ax = A + s.p;
  const unsigned int* By = B + s.q;
  const int per = (j + nt - 1) / nt;
  const int i0 = min(j, t * per), i1 = min(j, i0 + per);
  if (i0 >= i1) return;
  const int k0 = 2 * i0;
  int lo = max(0, k0 - y), hi = min(k0, x);
  while (lo < hi) {
    const int a = (lo + hi) >> 1;
    const int b = k0 - a;
    if (b > 0 && a < x && By[b - 1] >= Ax[a]) lo = a + 1;
    else hi = a;
  }
  int a = lo, b = k0 - lo;
  const unsigned int base = (unsigned int)(n + s.nb);
  for (int i = i0; i < i1; ++i) {
    unsigned int wsum = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const bool leaf = b >= y || (a < x && Ax[a] <= By[b]);
      const unsigned int id = leaf ? (unsigned int)(s.p + a) : (unsigned int)(n + s.q + b);
      wsum += leaf ? Ax[a] : By[b];
      parent[id] = base + (unsigned int)i;
      if (leaf) ++a; else ++b;
    }
    B[s.nb + i] = wsum;
  }
}

// Returns the number of rounds; rstart[r] is the first node id made in round r.
// Warp 0 runs rounds of at most kWarpJoin pairs on its own (no block-wide
// barrier); a larger round is joined by the whole block.
constexpr int kWarpJoin = 256;

__device__ int huff_two_queue(const unsigned int* A, unsigned int* B, int n, unsigned int* parent, int* rstart,
                              TwoQ* s, int* s_flag) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    s->p = 0;
    s->q = 0;
    s->nb = 0;
    s_flag[0] = 0;  // done
    s_flag[1] = 0;  // rounds
  }
  __syncthreads();
  while (true) {
    if (tid < 32) {
      while (true) {
        if ((n - s->p) + (s->nb - s->q) <= 1) {
          if (tid == 0) s_flag[0] = 1;
          break;
        }
        two_queue_plan(A, B, n, s);
        __syncwarp();
        const TwoQ c = *s;
        if (c.j > kWarpJoin) break;
        if (tid == 0) rstart[s_flag[1]] = n + c.nb;
        two_queue_join(A, B, n, c, parent, tid, 32);
        __syncwarp();
        if (tid == 0) {
          s->p = c.p + c.x;
          s->q = c.q + 2 * c.j - c.x;
          s->nb = c.nb + c.j;
          s_flag[1] += 1;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (s_flag[0]) break;
    const TwoQ c = *s;
    if (tid == 0) rstart[s_flag[1]] = n + c.nb;
    two_queue_join(A, B, n, c, parent, tid, blockDim.x);
    __syncthreads();
    if (tid == 0) {
      s->p = c.p + c.x;
      s->q = c.q + 2 * c.j - c.x;
      s->nb = c.nb + c.j;
      s_flag[1] += 1;
    }
    __syncthreads();
  }
  return s_flag[1];
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
  __shared__ unsigned int s_lend[32];
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
  // largest count -> number of 4-bit radix passes
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  if ((tid & 31) == 0) s_scan[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    unsigned long long m2 = 0;
    for (int i = 0; i < 32; ++i) m2 = max(m2, s_scan[i]);
    int np = 0;
    while (np < 8 && (m2 >> (4 * np)) != 0) ++np;
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
      if (lens) {  // absent when only the list is wanted
        lens[s] = 1;
        cw[s] = 1u << 24;
      }
      st_u32(out + off_cb, s | (1u << 16));
    }
    for (unsigned long long i = off_cb + 4ull * n + tid; i < off_bb; i += nt) out[i] = 0;
    return;
  }
  // leaves sorted by (count, symbol): stable sort by count of the symbol-ordered list
  unsigned int* ks;
  uint16_t* vs;
  {
    unsigned short* s_cnt = reinterpret_cast<unsigned short*>(arena);
    unsigned int* sk0 = reinterpret_cast<unsigned int*>(arena + 16 * kCbThreads * sizeof(unsigned short));
    unsigned int* sk1 = sk0 + kSegN;
    uint16_t* sv0 = reinterpret_cast<uint16_t*>(sk1 + kSegN);
    uint16_t* sv1 = sv0 + kSegN;
    ks = reinterpret_cast<unsigned int*>(hs.la);
    vs = reinterpret_cast<uint16_t*>(hs.lb);
    if (n <= kSegN) {
      for (int i = tid; i < n; i += nt) {
        sk0[i] = kc[i];
        sv0[i] = vc[i];
      }
      __syncthreads();
      smem_sort(sk0, sv0, sk1, sv1, n, s_u[1], ks, vs, s_cnt, s_scan);
    } else {
      // in the workspace, 8-bit digits
      unsigned int* qk = reinterpret_cast<unsigned int*>(hs.depth);
      uint16_t* qv = reinterpret_cast<uint16_t*>(qk + nsym);
      cta_radix_sort8(kc, vc, kc + nsym, vc + nsym, qk, qv, ks, vs, n, (s_u[1] + 1) / 2,
                      reinterpret_cast<unsigned int*>(arena), s_scan);
    }
  }
  for (int i = tid; i < 128; i += nt) s_bits[i] = 0;
  // merge rounds on the two queues: in shared memory when both fit, else the
  // internal-node queue alone (the leaves are read-only and stay in the workspace)
  unsigned int* parent = reinterpret_cast<unsigned int*>(hs.parent);
  const unsigned int* qa = ks;
  unsigned int* qb = reinterpret_cast<unsigned int*>(hs.w);
  if (n <= kCbQueueN) {
    unsigned int* sA = reinterpret_cast<unsigned int*>(arena);
    for (int i = tid; i < n; i += nt) sA[i] = ks[i];
    qa = sA;
    qb = sA + kCbQueueN;
  } else if ((size_t)n * 4 <= kCbSmem) {
    qb = reinterpret_cast<unsigned int*>(arena);
  }
  __shared__ TwoQ s_q;
  const int rounds = huff_two_queue(qa, qb, n, parent, hs.rstart, &s_q, &s_u[2]);
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
      st->cb_first[l] = code;
      st->cb_offs[l] = off;
    }
  }
  __syncthreads();
  const int maxlen = s_u[0];
  // canonical order: most frequent first (the sorted leaf list reversed);
  // the code tables indexed by symbol are filled by k_cb_assign
#pragma unroll 4
  for (int i = tid; i < n; i += nt) {
    const unsigned int leaf = (unsigned int)(n - 1 - i);
    // length = largest l with leaf < s_lend[l] (s_lend decreases with l)
    int lo2 = 1, hi2 = maxlen;
    while (lo2 < hi2) {
      const int mid = (lo2 + hi2 + 1) >> 1;
      if (leaf < s_lend[mid]) lo2 = mid; else hi2 = mid - 1;
    }
    st_u32(out + off_cb + 4ull * i, (unsigned int)vs[leaf] | ((unsigned int)lo2 << 16));
  }
  for (unsigned long long i = off_cb + 4ull * n + tid; i < off_bb; i += nt) out[i] = 0;
}

// Length and code word of every used symbol, from the ordered codebook
// section: entry i of length l has code cb_first[l] + (i - cb_offs[l]).
// Many CTAs, so the writes scattered by symbol spread over the GPU.
__global__ void __launch_bounds__(256) k_cb_assign(const uint8_t* __restrict__ out, uint8_t* lens, uint32_t* cw,
                                                   const State* __restrict__ st) {
  if (st->err) return;
  const unsigned int n = st->n_used;
  const unsigned int i = blockIdx.x * 256u + threadIdx.x;
  if (n <= 1 || i >= n) return;
  const unsigned int e = *reinterpret_cast<const unsigned int*>(out + st->off_cb + 4ull * i);
  const unsigned int sym = e & 0xFFFFu, l = e >> 16;
  lens[sym] = (uint8_t)l;
  cw[sym] = (st->cb_first[l] + (i - st->cb_offs[l])) | (l << 24);
}

int launch_codebook(const unsigned long long* hist, int m, uint8_t* lens, uint32_t* cw, State* st,
                    const HuffScratch& hs, uint8_t* out, const Geo& g, const HdrInfo& hi, cudaStream_t s) {
  const size_t smem = kCbSmem;
  if (cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PC_ERR_CUDA;
  ProfScope p(kStCodebook, s);
  k_codebook<<<1, kCbThreads, smem, s>>>(hist, m, lens, cw, st, hs, out, (unsigned long long)g.nblocks, hi.off_cb,
                                         hi.cap);
  k_cb_assign<<<((1u << m) + 255u) / 256u, 256, 0, s>>>(out, lens, cw, st);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

// Code table of a given codebook list (the sample codebook of the training
// phase, already copied into the container's codebook section, checked on the
// host: lengths 1..24 never decreasing, distinct symbols, Kraft sum <= 1).
// One CTA: clear the table, count the entries per length, then each entry i
// of length l gets the canonical code first[l] + (i - offs[l]).
__global__ void __launch_bounds__(1024) k_cb_table(const uint8_t* __restrict__ out, unsigned long long off_cb, int n,
                                                   int m, uint32_t* cwl, State* st, unsigned long long nblocks,
                                                   unsigned long long cap) {
  __shared__ unsigned int s_cnt[32], s_first[32], s_offs[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < 32) s_cnt[tid] = 0u;
  for (int i = tid; i < (1 << m); i += nt) cwl[i] = 0u;
  __syncthreads();
  const unsigned int* list = reinterpret_cast<const unsigned int*>(out + off_cb);
  for (int i = tid; i < n; i += nt) atomicAdd(&s_cnt[(list[i] >> 16) & 31u], 1u);
  __syncthreads();
  if (tid == 0) {
    unsigned int code = 0, off = 0;
    for (int l = 1; l <= kLmax; ++l) {
      const unsigned int prevc = l > 1 ? s_cnt[l - 1] : 0u;
      code = (code + prevc) << 1;
      off += prevc;
      s_first[l] = code;
      s_offs[l] = off;
    }
    const unsigned long long off_bb = al16(off_cb + 4ull * (unsigned long long)n);
    const unsigned long long off_bn = al16(off_bb + 4ull * nblocks);
    st->n_used = (unsigned int)n;
    st->off_cb = off_cb;
    st->off_bb = off_bb;
    st->off_bn = off_bn;
    if (off_bn + 2ull * nblocks > cap) st->err = PC_ERR_CAPACITY;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const unsigned int e = list[i];
    const unsigned int sym = e & 0xFFFFu, l = e >> 16;
    cwl[sym] = (s_first[l] + ((unsigned int)i - s_offs[l])) | (l << 24);
  }
}

int launch_cb_table(const uint8_t* out, unsigned long long off_cb, int n, int m, uint32_t* cwl, State* st,
                    const Geo& g, unsigned long long cap, cudaStream_t s) {
  ProfScope p(kStCodebook, s);
  k_cb_table<<<1, 1024, 0, s>>>(out, off_cb, n, m, cwl, st, (unsigned long long)g.nblocks, cap);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

int launch_huff_list(const unsigned long long* hist, int m, State* st, const HuffScratch& hs, uint8_t* list,
                     unsigned long long cap, cudaStream_t s) {
  const size_t smem = kCbSmem;
  if (cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PC_ERR_CUDA;
  // no lengths or code tables, no block table: the list at offset 0
  k_codebook<<<1, kCbThreads, smem, s>>>(hist, m, nullptr, nullptr, st, hs, list, 0ull, 0ull, cap);
  return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // namespace pc
