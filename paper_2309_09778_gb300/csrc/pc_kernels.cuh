// Declarations shared by the kernel translation units and the C-ABI layer.
#pragma once
#include "pc_device.cuh"

namespace pc {

// Field and block geometry.
struct Geo {
  long long n[3];    // field dims, n[2] fastest
  int b[3];          // block shape
  long long nb[3];   // blocks per axis
  long long nblocks;
  int bvol;          // b[0]*b[1]*b[2]
  int ch;            // blocks per pack/decode chunk
  long long nchunks;
};

// Bricks: a CTA of 256 threads handles G consecutive blocks along x, one
// team of 256/G threads per block, at most 4096 points per brick.
template <int BV>
struct BrickShape {
  static constexpr int G = BV <= 512 ? 8 : (BV <= 1024 ? 4 : (BV <= 2048 ? 2 : 1));
  static constexpr int TS = 256 / G;
  static constexpr int PPT = (BV + TS - 1) / TS;
};

// Block with a zero border: stencil neighbours outside the block read 0
// without bounds checks.  WIDE adds the +1 border in y and x that the
// 13-point stencil reaches.  The pitches keep one spare row and column beyond
// the border: with pitches B + 1 (B + 2 when WIDE) the points of one
// reconstruction wavefront (the plane z + y + x = s or 4z + 2y + x = s) fall
// on a few shared-memory banks (8-way conflicts for 8^3 blocks); the extra
// pitch spreads them over all 32.
template <int B0, int B1, int B2, bool WIDE>
struct Pad {
  static constexpr int P1 = B1 + (WIDE ? 3 : 2);
  static constexpr int P2 = B2 + (WIDE ? 3 : 2);
  static constexpr int PV = (B0 + 1) * P1 * P2;
  static __device__ __forceinline__ int at(int lz, int ly, int lx) { return ((lz + 1) * P1 + (ly + 1)) * P2 + (lx + 1); }
  static constexpr int off(int dz, int dy, int dx) { return (dz * P1 + dy) * P2 + dx; }
};

template <int TS>
__device__ __forceinline__ int team_sum(int v, int* slot) {
  if constexpr (TS == 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
  } else {
    atomicAdd(slot, v);
    return 0;  // caller reads *slot after a barrier
  }
}

// Values the header needs that only the host knows.
struct HdrInfo {
  int dtype, pred, stencil, h1, h2, m, s_in, nw;
  int wsz;                    // bytes per weights-section entry: 4 (f32 weights) or 8 (int64 fixed-point network)
  unsigned int flags;         // header flags (kFlagStreamFirst, kFlagLiteral)
  int eq_period;              // literal selection: equilibrium-point period (header offset 232)
  double eb;
  unsigned long long off_cb;  // = al16(256 + wsz nw)
  unsigned long long cap;     // output capacity in bytes
};

// Huffman construction scratch (all in the caller's workspace).
struct HuffScratch {
  unsigned long long* key;   // [np2] sort keys
  unsigned long long* w;     // [2 nsym] node weights
  int* parent;               // [2 nsym]
  int* depth;                // [2 nsym]
  int* la;                   // [nsym] node list
  int* lb;                   // [nsym] node list
  int* rstart;               // [nsym + 2] first node id of each merge round
  unsigned int* symord;      // [nsym] used symbols in symbol order
};

// Block-wide exclusive scan (any blockDim multiple of 32, up to 1024); total
// receives the block sum.  Contains __syncthreads: call from every thread.
template <typename V>
__device__ __forceinline__ V cta_exscan(V v, V* s_w, V& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  V x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    V y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    V t = lane < nw ? s_w[lane] : (V)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      V y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  V pre = (w > 0 ? s_w[w - 1] : (V)0) + x - v;
  total = s_w[nw - 1];
  __syncthreads();
  return pre;
}

__device__ __forceinline__ void st_u32(uint8_t* p, unsigned int v) { *reinterpret_cast<unsigned int*>(p) = v; }
__device__ __forceinline__ void st_u64(uint8_t* p, unsigned long long v) {
  *reinterpret_cast<unsigned long long*>(p) = v;
}

__host__ __device__ inline unsigned long long al16(unsigned long long x) { return (x + 15ull) & ~15ull; }

template <typename T>
int launch_stats_consts(const void* x, unsigned long long n, State* st, Tabs* tabs, unsigned long long* hist,
                        int nsym, double eb, int nsm, cudaStream_t s);
// Container flag (header offset 228): the bitstream precedes the balance
// values, the layout that single-pass compression writes.
constexpr unsigned int kFlagStreamFirst = 1u;
// Container flag: codes of the paper-literal data selection (Section IV.D;
// decoded with drift); header offset 232 holds the equilibrium-point period.
constexpr unsigned int kFlagLiteral = 4u;
// Container flag: the bitstream section holds the lossless stage's chunks
// (header offset 240: the section's bytes).
constexpr unsigned int kFlagLossless = 8u;
constexpr int kLzChunk = 16384;             // bytes per chunk of the lossless stage
constexpr int kLzSlot = kLzChunk + 256;     // workspace bytes per chunk's tokens
// Workspace of the lossless stage: per chunk a token slot, its size and its
// section offset; nch_max chunks (the longest stream).
struct LzBufs {
  uint8_t* slots;
  unsigned int* sizes;
  unsigned long long* offs;
  unsigned long long nch_max;
};
unsigned long long lz_chunks_max(unsigned long long raw_max);
// The stage over the finished stream (its offset and length in the state):
// the container's stream section replaced by the chunks, header rewritten.
int launch_lz_encode(uint8_t* out, unsigned long long cap, State* st, const LzBufs& lb, cudaStream_t s);
// The raw stream (nraw bytes) back from a section of lzb bytes (offs: one
// u64 per chunk of scratch).
int launch_lz_decode(const uint8_t* sec, unsigned long long lzb, unsigned long long nraw, uint8_t* raw,
                     unsigned long long* offs, int* err, cudaStream_t s);

// Bricks of a field: G blocks along x per brick (BrickShape), rows of bricks.
inline long long bricks_of(const Geo& g) {
  const int G = g.bvol <= 512 ? 8 : (g.bvol <= 1024 ? 4 : (g.bvol <= 2048 ? 2 : 1));
  return g.nb[0] * g.nb[1] * ((g.nb[2] + G - 1) / G);
}

// One field of a fused compression launch: its input, geometry, per-call
// state (constants, tables, histogram) and outputs.  brick0 is the field's
// first brick in the launch's brick numbering (fields in order).
struct CJob {
  const void* x;
  Geo g;
  const State* st;
  const Tabs* tabs;
  uint16_t* codes;
  uint8_t* nnflag;
  uint32_t* nout;
  unsigned long long* hist;
  const long long* qnet;  // fixed-point network (container weights section) or null
  long long brick0;
  int m;
  int pad_;
  // single pass (a given codebook): the container, the code table, the
  // look-back records, each brick's first and last stream word, and the
  // balance values in container order (workspace)
  uint8_t* out;
  const uint32_t* cwl;       // [2^m] (length << 24) | code word; 0 for symbols outside the codebook
  unsigned long long* rec;   // [2 nbk]: bit counts, then balance-point counts (flag << 62 | value)
  uint32_t* side;            // [2 nbk]
  void* ov;                  // [points] balance values
  unsigned long long off_bb, off_bn, off_st;
  unsigned long long cap_words;  // stream words that fit the output
  long long nbk;             // bricks of the field
};
constexpr int kMaxJobs = 32;  // fields per fused launch (the table travels as a kernel parameter)
struct CJobs {
  int n;
  int pad_;
  long long total;  // bricks of all fields
  // single pass: bricks are taken in order from this counter (zeroed before
  // the launch), so that every brick a look-back waits for belongs to a
  // running CTA; null: static assignment, no look-back
  unsigned long long* next;
  CJob j[kMaxJobs];
};

// Compression of n fields that share dtype, block shape and predictor form
// (and, for the FP32 perceptron, the weights mlp) in one persistent launch;
// with `next`, single-pass packing against each job's codebook.
template <typename T>
int launch_compress(const CJob* jobs, int n, int mode, const Mlp& mlp, int nsm, cudaStream_t s,
                    unsigned long long* next = nullptr);
// Code table of a given codebook list (already in the container at off_cb):
// cwl[sym] = (length << 24) | canonical code word, 0 for absent symbols; sets
// the codebook and block-table offsets in the state.
int launch_cb_table(const uint8_t* out, unsigned long long off_cb, int n, int m, uint32_t* cwl, State* st,
                    const Geo& g, unsigned long long cap, cudaStream_t s);
// Finish of a single-pass compression: stream words shared by bricks, the
// balance values moved after the stream, section pads, weights and header.
struct SpFinish {
  const unsigned long long* rec;
  const uint32_t* side;
  const void* ov;
  long long nbk;
  unsigned long long off_bb, off_bn, off_st;
};
template <typename T>
int launch_sp_finish(const Geo& g, State* st, uint8_t* out, const HdrInfo& hi, const Mlp& mlp, const SpFinish& f,
                     int nsm, cudaStream_t s);
int launch_codebook(const unsigned long long* hist, int m, uint8_t* lens, uint32_t* cw, State* st,
                    const HuffScratch& hs, uint8_t* out, const Geo& g, const HdrInfo& hi, cudaStream_t s);
template <typename T>
int launch_pack(const T* x, const Geo& g, const uint16_t* codes, const uint8_t* nnflag, const uint32_t* nout,
                const uint8_t* lens, const uint32_t* cw, uint32_t* bbits, unsigned long long* chunk_bits,
                unsigned long long* chunk_nout, unsigned long long* chunk_boff, unsigned long long* chunk_ooff,
                State* st, uint8_t* out, const HdrInfo& hi, const Mlp& mlp, cudaStream_t s);

// Decompression.
struct DecInfo {
  int dtype, m, stencil, h1, h2, s_in, usenn_any, qmode;
  int literal;            // codes of the paper-literal data selection (float32 only)
  const uint8_t* stream;  // the bitstream words: in the container, or decoded from the lossless stage
  const long long* qnet;  // fixed-point network in the container (qmode), else null
  unsigned int n_used;
  unsigned long long n_out, swords;
  unsigned long long off_cb, off_bb, off_bn, off_ov, off_st, in_size;
  int Kp, Kn, Zq, S;
  unsigned long long step_bits, inv_bits, ebdn_bits;
};
struct DecScratch {
  uint16_t* sorted;            // [2^m] symbols in code order (the stored codebook list)
  unsigned int* tabs;          // [3 * 32]: first code, count, offset per length
  unsigned long long* chunk_bits;
  unsigned long long* chunk_nout;
  unsigned long long* chunk_boff;
  unsigned long long* chunk_ooff;
  unsigned long long* boff;    // [nblocks]
  unsigned long long* ooff;    // [nblocks]
  uint16_t* codes;             // [nblocks * bvol]
  Tabs* ftab;                  // log2 / 2^t tables
  int* err;                    // device error word
};
// Training buffers (all in the caller's workspace).
struct TrainBufs {
  unsigned int *cnt_t, *cnt_v;
  unsigned long long *off_t, *off_v;
  int *tin, *ttg, *vin, *vtg;
  uint8_t *tus, *vus;
  float* w;
  const float *lrs, *lams;
  unsigned long long* costs;
  void* ctl;
  unsigned long long cap_t, cap_v;
};
size_t train_ctl_bytes();
// Buffers of the selection by simulated compression: per-model code
// histograms (u64 [nmodels + 1][2^m]) and residual bit-length counts
// (u64 [nmodels + 1][34]), a scratch state, codebook list and Huffman scratch.
struct SelectBufs {
  unsigned long long* hists;
  unsigned long long* bitcnt;
  State* st;
  uint8_t* list;
  HuffScratch hs;
};
// Score the trained models and Lorenzo by simulated compression into
// tb.costs and choose (Lorenzo unless strictly beaten).
int launch_select(const TrainBufs& tb, const SelectBufs& sb, int k, int h1, int h2, int m, int nmodels,
                  int value_bits, cudaStream_t s);
// Huffman code lengths of one histogram as a codebook list (sym | len << 16,
// most frequent first) at list[0..], n_used in st (a zeroed scratch state).
int launch_huff_list(const unsigned long long* hist, int m, State* st, const HuffScratch& hs, uint8_t* list,
                     unsigned long long cap, cudaStream_t s);
// The sample codebook of the training phase (validation samples of seed and
// thr32, residuals of the FP32 weights in tb.w[0] or of Lorenzo, at m code
// bits; span_fill: every code inside the sampled span coded) as a codebook
// list in sb.list, its length in sb.st->n_used.
template <typename T>
int launch_sample_hist(const T* x, const Geo& g, const State* st, const Tabs* tabs, const TrainBufs& tb,
                       const SelectBufs& sb, int k, int h1, int h2, int s_in, int m, bool lorenzo, int span_fill,
                       unsigned long long seed, unsigned int thr32, cudaStream_t s);
template <typename T>
int launch_train(const T* x, const Geo& g, const State* st, const Tabs* tabs, const TrainBufs& tb, int k, int h1,
                 int h2, int m, int nmodels, unsigned long long seed, unsigned int thr32, cudaStream_t s);

template <typename T>
int launch_quantize(const T* x, const Geo& g, const State* st, const Tabs* tabs, const TrainBufs& tb, int k, int h1,
                    int h2, int s_in, unsigned long long seed, unsigned int thr32, long long* q,
                    unsigned long long* qmax, cudaStream_t s);

// Host destination of a decompression that copies the field out slab by slab
// (whole block planes) on its own stream while later slabs are reconstructed;
// `used` tells whether the reconstruction took that path (else the caller
// copies the whole field).
constexpr int kSlabs = 8;
struct SlabSink {
  void* host;
  cudaStream_t cs;
  cudaEvent_t ev[kSlabs + 1];
  bool used;
};
// Phases of a decompression: everything, only what precedes the Huffman
// decoder (checks, tables, offsets), or only what follows it (reconstruction).
constexpr int kDecAll = 0, kDecPrep = 1, kDecRecon = 2;
template <typename T>
int launch_decompress(const uint8_t* in, const Geo& g, const DecInfo& di, const DecScratch& ds, const Mlp& mlp,
                      T* out, int nsm, cudaStream_t s, SlabSink* sink = nullptr, int phase = kDecAll);
// One field of a fused Huffman-decoder launch; cta0 is its first CTA.
struct DecJob {
  Geo g;
  const uint8_t* in;
  DecInfo di;
  DecScratch ds;
  long long cta0;
};
constexpr int kMaxDecJobs = 32;
struct DecJobs {
  int n;
  int pad_;
  DecJob j[kMaxDecJobs];
};
// The Huffman decoder of n fields (each prepared by a kDecPrep phase) in one launch.
int launch_huff_jobs(const DecJob* jobs, int n, cudaStream_t s);
// The paper-literal data selection (Section IV.D, float32): codes, flags,
// balance counts and histogram of a field (mode 0 Lorenzo, 1 FP32 perceptron);
// and the drifting decoder that follows the Huffman decoder.
int launch_lit_compress(const float* x, const Geo& g, const State* st, const Tabs* tabs, const Mlp& mlp, int mode,
                        int eq_period, int m, uint16_t* codes, uint8_t* nnflag, uint32_t* nout,
                        unsigned long long* hist, int nsm, cudaStream_t s);
int launch_lit_decode(const uint8_t* in, const Geo& g, const DecInfo& di, const DecScratch& ds, const Mlp& mlp,
                      float* out, int nsm, cudaStream_t s);

}  // namespace pc
