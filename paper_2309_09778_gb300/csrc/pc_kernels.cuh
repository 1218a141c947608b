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

// Values the header needs that only the host knows.
struct HdrInfo {
  int dtype, pred, stencil, h1, h2, m, s_in, nw;
  double eb;
  unsigned long long off_cb;  // = al16(256 + 4 nw)
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
int launch_stats_consts(const void* x, unsigned long long n, State* st, unsigned long long* hist, int nsym,
                        double eb, int nsm, cudaStream_t s);
template <typename T>
int launch_compress(const void* x, const Geo& g, const State* st, uint16_t* codes, uint8_t* nnflag, uint32_t* nout,
                    unsigned long long* hist, int m, int mode, const Mlp& mlp, int nsm, cudaStream_t s);
int launch_codebook(const unsigned long long* hist, int m, uint8_t* lens, uint32_t* cw, State* st,
                    const HuffScratch& hs, uint8_t* out, const Geo& g, const HdrInfo& hi, cudaStream_t s);
template <typename T>
int launch_pack(const T* x, const Geo& g, const uint16_t* codes, const uint8_t* nnflag, const uint32_t* nout,
                const uint8_t* lens, const uint32_t* cw, uint32_t* bbits, unsigned long long* chunk_bits,
                unsigned long long* chunk_nout, unsigned long long* chunk_boff, unsigned long long* chunk_ooff,
                State* st, uint8_t* out, const HdrInfo& hi, const Mlp& mlp, cudaStream_t s);

// Decompression.
struct DecInfo {
  int dtype, m, stencil, h1, h2, s_in, usenn_any;
  unsigned int n_used;
  unsigned long long n_out, swords;
  unsigned long long off_cb, off_bb, off_bn, off_ov, off_st, in_size;
  int Kp, Kn, Zq, S;
  unsigned long long step_bits, inv_bits, ebdn_bits;
};
struct DecScratch {
  uint8_t* lens;               // [2^m]
  uint16_t* sorted;            // [2^m] symbols in canonical (length, symbol) order
  unsigned int* lut;           // [4096] 12-bit first-level decode table
  unsigned int* tabs;          // [3 * 32]: first code, count, offset per length
  unsigned long long* key;     // [np2] sort scratch
  unsigned long long* chunk_bits;
  unsigned long long* chunk_nout;
  unsigned long long* chunk_boff;
  unsigned long long* chunk_ooff;
  unsigned long long* boff;    // [nblocks]
  unsigned long long* ooff;    // [nblocks]
  uint16_t* codes;             // [nblocks * bvol]
  int* err;                    // device error word
};
template <typename T>
int launch_decompress(const uint8_t* in, const Geo& g, const DecInfo& di, const DecScratch& ds, const Mlp& mlp,
                      T* out, int nsm, cudaStream_t s);

}  // namespace pc
