// C ABI (include/pc.h): argument checks, workspace layout, launch sequence.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "pc_kernels.cuh"
#include "pc_qmlp.cuh"
#include "pc_profile.cuh"

using namespace pc;

namespace {

constexpr size_t kAlign = 256;
inline size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64) cache[dev] = n;
  return n;
}

bool shape_supported(const int b[3]) {
  static const int shapes[][3] = {{8, 8, 8}, {4, 4, 4}, {16, 16, 16}, {1, 16, 32}, {1, 8, 8}, {1, 64, 64}};
  for (auto& s : shapes)
    if (s[0] == b[0] && s[1] == b[1] && s[2] == b[2]) return true;
  return false;
}

int nweights(int k, int h1, int h2) {
  const int hl = h2 > 0 ? h2 : h1;
  return h1 * k + h1 + (h2 > 0 ? h2 * h1 + h2 : 0) + hl + 1;
}

bool make_geo(const size_t dims[3], const int block[3], Geo& g) {
  long long vol = 1;
  for (int i = 0; i < 3; ++i) {
    if (dims[i] < 1 || dims[i] > 0xFFFFFFFFull || block[i] < 1) return false;
    g.n[i] = (long long)dims[i];
    g.b[i] = block[i];
    g.nb[i] = (g.n[i] + block[i] - 1) / block[i];
    vol *= block[i];
  }
  if (vol < 2 || vol > 4096) return false;
  // Huffman weights are 32-bit counts of points
  if ((unsigned long long)g.n[0] * (unsigned long long)g.n[1] > 0xFFFFFFFFull ||
      (unsigned long long)g.n[0] * (unsigned long long)g.n[1] * (unsigned long long)g.n[2] > 0xFFFFFFFFull)
    return false;
  g.bvol = (int)vol;
  g.nblocks = g.nb[0] * g.nb[1] * g.nb[2];
  long long ch = kChunkPts / g.bvol;
  if (ch < 1) ch = 1;
  if (ch > 1024) ch = 1024;
  g.ch = (int)ch;
  g.nchunks = (g.nblocks + ch - 1) / ch;
  return true;
}

bool qshape_ok(int k, int h1, int h2) { return (k == 7 && h1 == 16 && h2 == 16) || (k == 13 && h1 == 32 && h2 == 32); }

bool train_shape_ok(int k, int h1, int h2);

// The predictor is trained inside pc_compress (no weights given).
// A given codebook list (sym | length << 16, in container order): at most
// 2^m entries, symbols below 2^m and distinct, lengths 1..24 never decreasing
// (the canonical construction runs along the list), Kraft sum at most one,
// symbol 0 present (balance points are coded as symbol 0), and a single
// entry of length 1.
bool codebook_ok(const unsigned int* cb, int n, int m) {
  const int nsym = 1 << m;
  if (n < 1 || n > nsym) return false;
  static thread_local uint8_t seen[1 << 16];
  memset(seen, 0, (size_t)nsym);
  unsigned long long kraft = 0;  // in units of 2^-24
  int prev = 1;
  bool have0 = false;
  for (int i = 0; i < n; ++i) {
    const unsigned int sym = cb[i] & 0xFFFFu, l = cb[i] >> 16;
    if (sym >= (unsigned int)nsym || l < 1 || l > (unsigned int)kLmax || (int)l < prev || seen[sym]) return false;
    if (n == 1 && l != 1) return false;
    seen[sym] = 1;
    prev = (int)l;
    kraft += 1ull << (kLmax - l);
    have0 |= sym == 0;
  }
  return have0 && kraft <= (1ull << kLmax);
}

// Bytes of the longest bitstream of n points (every code at the length limit).
unsigned long long stream_bytes_max(unsigned long long n) { return 4ull * ((n * kLmax + 31) / 32 + 1); }

bool wants_training(const pc_params* p) {
  return (p->pred == PC_PRED_MLP_FP32 && !p->h_weights) || (p->pred == PC_PRED_MLP_BF16 && !p->h_qnet);
}

int check_params(const size_t dims[3], int dtype, const pc_params* p, Geo& g, int& mode, int& nw) {
  if (!dims || !p) return PC_ERR_ARG;
  if (dtype != PC_F32 && dtype != PC_F64) return PC_ERR_DTYPE;
  if (!(p->eb_rel > 0.0 && p->eb_rel < 1.0)) return PC_ERR_ARG;
  if (p->m < 2 || p->m > 16) return PC_ERR_ARG;
  if (p->ndims < 0 || p->ndims > 3 || p->train_samples < 0) return PC_ERR_ARG;
  for (int i = 0; i < 3 - p->ndims && p->ndims > 0; ++i)
    if (dims[i] != 1) return PC_ERR_ARG;
  if (!make_geo(dims, p->block, g)) return PC_ERR_ARG;
  if (!shape_supported(p->block)) return PC_ERR_ARG;
  if (p->h_codebook && !codebook_ok(p->h_codebook, p->codebook_n, p->m)) return PC_ERR_ARG;
  // the paper-literal selection: float32, Lorenzo or the FP32 perceptron with weights, two passes
  if (p->literal && (dtype != PC_F32 || p->eq_period < 0 || p->h_codebook ||
                     (p->pred != PC_PRED_LORENZO && !(p->pred == PC_PRED_MLP_FP32 && p->h_weights))))
    return PC_ERR_ARG;
  if (!p->literal && p->eq_period != 0) return PC_ERR_ARG;
  if (p->lossless && p->h_codebook) return PC_ERR_ARG;  // the stage follows a stream that ends the container
  mode = p->pred == PC_PRED_MLP_FP32 ? 1 : (p->pred == PC_PRED_MLP_BF16 ? 2 : 0);
  if (p->pred != PC_PRED_LORENZO && p->pred != PC_PRED_MLP_FP32 && p->pred != PC_PRED_MLP_BF16) return PC_ERR_ARG;
  nw = 0;
  if (mode == 2) {
    if (!qshape_ok(p->stencil, p->hidden[0], p->hidden[1])) return PC_ERR_ARG;
    if (!p->h_qnet) return PC_OK;  // trained inside pc_compress
    if (p->s_in < 0 || p->s_in > 30) return PC_ERR_ARG;
    if (!qnet_valid(p->h_qnet, p->stencil, p->hidden[0], p->hidden[1], p->s_in)) return PC_ERR_ARG;
    nw = qnet_len(p->stencil, p->hidden[0], p->hidden[1]);
  } else if (mode) {
    if (p->stencil != 7 && p->stencil != 13) return PC_ERR_ARG;
    if (p->hidden[0] < 2 || p->hidden[0] > kMaxH || p->hidden[1] < 0 || p->hidden[1] > kMaxH) return PC_ERR_ARG;
    nw = nweights(p->stencil, p->hidden[0], p->hidden[1]);
    if (nw > kMaxW) return PC_ERR_ARG;
    if (!p->h_weights) {  // trained inside pc_compress
      if (!train_shape_ok(p->stencil, p->hidden[0], p->hidden[1])) return PC_ERR_ARG;
      return PC_OK;
    }
    if (p->s_in < 0 || p->s_in > 30) return PC_ERR_ARG;
  }
  return PC_OK;
}

struct CompLayout {
  size_t st, tabs, hist, lens, cw, key, w, parent, depth, la, lb, rstart, symord, codes, nnflag, nout, bbits, cbits, cnout,
      cboff, cooff, rec, side, next, ov, lzslot, lzsize, lzoff, total;
  unsigned long long lz_nch;
};

// sp: single pass (a given codebook): no code spill; look-back records, brick
// edge words, the brick counter and room for every point as a balance value
// (ts bytes each) instead.
CompLayout comp_layout(const Geo& g, int m, bool sp = false, size_t ts = 4, bool lossless = false) {
  const size_t nsym = (size_t)1 << m;
  size_t np = 1;
  while (np < nsym) np <<= 1;
  CompLayout L;
  size_t o = 0;
  L.st = o; o = up(o + sizeof(State));
  L.tabs = o; o = up(o + sizeof(Tabs));
  L.hist = o; o = up(o + 8 * nsym);
  L.lens = o; o = up(o + nsym);
  L.cw = o; o = up(o + 4 * nsym);
  L.key = o; o = up(o + 8 * np);
  L.w = o; o = up(o + 8 * 2 * nsym);
  L.parent = o; o = up(o + 4 * 2 * nsym);
  L.depth = o; o = up(o + 4 * 2 * nsym);
  L.la = o; o = up(o + 4 * nsym);
  L.lb = o; o = up(o + 4 * nsym);
  L.rstart = o; o = up(o + 4 * (nsym + 2));
  L.symord = o; o = up(o + 4 * nsym);
  L.codes = o; o = up(o + (sp ? 0 : 2 * (size_t)g.nblocks * g.bvol));
  L.nnflag = o; o = up(o + (size_t)g.nblocks);
  L.nout = o; o = up(o + 4 * (size_t)g.nblocks);
  L.bbits = o; o = up(o + 4 * (size_t)g.nblocks);
  L.cbits = o; o = up(o + 8 * (size_t)g.nchunks);
  L.cnout = o; o = up(o + 8 * (size_t)g.nchunks);
  L.cboff = o; o = up(o + 8 * (size_t)g.nchunks);
  L.cooff = o; o = up(o + 8 * (size_t)g.nchunks);
  const size_t nbk = sp ? (size_t)bricks_of(g) : 0;
  L.rec = o; o = up(o + 16 * nbk);
  L.side = o; o = up(o + 8 * nbk);
  L.next = o; o = up(o + (sp ? 16 : 0));
  L.ov = o; o = up(o + (sp ? ts * (size_t)g.n[0] * g.n[1] * g.n[2] : 0));
  // the lossless stage: per chunk of the longest stream a token slot, a size, an offset
  L.lz_nch = lossless ? lz_chunks_max(stream_bytes_max((unsigned long long)g.n[0] * g.n[1] * g.n[2])) : 0;
  L.lzslot = o; o = up(o + (size_t)kLzSlot * L.lz_nch);
  L.lzsize = o; o = up(o + 4 * (size_t)L.lz_nch);
  L.lzoff = o; o = up(o + 8 * (size_t)L.lz_nch);
  L.total = o;
  return L;
}

struct DecLayout {
  size_t err, ftab, sorted, tabs, cbits, cnout, cboff, cooff, boff, ooff, codes, lzraw, lzoff, total;
};

// lz_raw: bytes of the bitstream to decode from the lossless stage (0: none)
DecLayout dec_layout(const Geo& g, int m, unsigned long long lz_raw = 0) {
  const size_t nsym = (size_t)1 << m;
  DecLayout L;
  size_t o = 0;
  L.err = o; o = up(o + 16);
  L.ftab = o; o = up(o + sizeof(Tabs));
  L.sorted = o; o = up(o + 2 * nsym);
  L.tabs = o; o = up(o + 4 * 96);
  L.cbits = o; o = up(o + 8 * (size_t)g.nchunks);
  L.cnout = o; o = up(o + 8 * (size_t)g.nchunks);
  L.cboff = o; o = up(o + 8 * (size_t)g.nchunks);
  L.cooff = o; o = up(o + 8 * (size_t)g.nchunks);
  L.boff = o; o = up(o + 8 * (size_t)g.nblocks);
  L.ooff = o; o = up(o + 8 * (size_t)g.nblocks);
  L.codes = o; o = up(o + 2 * (size_t)g.nblocks * g.bvol);
  L.lzraw = o; o = up(o + (lz_raw ? al16(lz_raw) + 64 : 0));
  L.lzoff = o; o = up(o + 8 * (size_t)lz_chunks_max(lz_raw));
  L.total = o;
  return L;
}

// CRC-32 (IEEE 802.3, reflected) for header validation on the host.
uint32_t host_crc32(const uint8_t* p, size_t n) {
  static uint32_t table[256];
  static std::once_flag once;
  std::call_once(once, [] {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? (0xEDB88320u ^ (c >> 1)) : (c >> 1);
      table[i] = c;
    }
  });
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) c = table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
  return c ^ 0xFFFFFFFFu;
}

uint32_t rd32(const uint8_t* p) { uint32_t v; memcpy(&v, p, 4); return v; }
uint64_t rd64(const uint8_t* p) { uint64_t v; memcpy(&v, p, 8); return v; }

// Parsed, validated header.
struct Hdr {
  int dtype, pred, m, stencil, h1, h2, s_in, nw, block[3];
  int literal, lossless;
  unsigned long long lzb;
  size_t dims[3];
  unsigned int n_used;
  unsigned long long nblocks, n_out, swords, off_cb, off_bb, off_bn, off_ov, off_st, total;
  int Kp, Kn, Zq, S;
  unsigned long long step_bits, inv_bits, ebdn_bits;
};

int parse_header(const uint8_t* h, size_t n, Hdr& H, Geo& g) {
  if (!h || n < (size_t)kHdr) return PC_ERR_CORRUPT;
  if (rd32(h) != 0x504D4350u || rd32(h + 4) != 1u) return PC_ERR_CORRUPT;
  if (rd32(h + 252) != host_crc32(h, 252)) return PC_ERR_CORRUPT;
  H.dtype = (int)rd32(h + 8);
  H.pred = (int)rd32(h + 12);
  for (int i = 0; i < 3; ++i) {
    H.dims[i] = (size_t)rd64(h + 16 + 8 * i);
    H.block[i] = (int)rd32(h + 40 + 4 * i);
  }
  H.stencil = (int)rd32(h + 52);
  H.h1 = (int)rd32(h + 56);
  H.h2 = (int)rd32(h + 60);
  H.m = (int)rd32(h + 64);
  H.s_in = (int)rd32(h + 68);
  H.Kp = (int)rd32(h + 100);
  H.Kn = (int)rd32(h + 104);
  H.Zq = (int)rd32(h + 108);
  H.S = (int)rd32(h + 112);
  H.n_used = rd32(h + 116);
  H.step_bits = rd64(h + 120);
  H.inv_bits = rd64(h + 128);
  H.ebdn_bits = rd64(h + 136);
  H.nblocks = rd64(h + 144);
  H.n_out = rd64(h + 152);
  H.swords = rd64(h + 160);
  H.off_cb = rd64(h + 176);
  H.off_bb = rd64(h + 184);
  H.off_bn = rd64(h + 192);
  H.off_ov = rd64(h + 200);
  H.off_st = rd64(h + 208);
  H.total = rd64(h + 216);
  H.nw = (int)rd32(h + 224);
  const unsigned int flags = rd32(h + 228);
  if (flags & ~(kFlagStreamFirst | kFlagLiteral | kFlagLossless)) return PC_ERR_CORRUPT;
  H.lossless = (flags & kFlagLossless) != 0;
  H.lzb = rd64(h + 240);
  if (H.lossless && (flags & kFlagStreamFirst)) return PC_ERR_CORRUPT;
  H.literal = (flags & kFlagLiteral) != 0;
  if (H.literal && (H.dtype != PC_F32 || (H.pred != 0 && H.pred != 1) || (flags & kFlagStreamFirst)))
    return PC_ERR_CORRUPT;
  if (H.dtype != PC_F32 && H.dtype != PC_F64) return PC_ERR_CORRUPT;
  if (H.m < 2 || H.m > 16) return PC_ERR_CORRUPT;
  for (int i = 0; i < 3; ++i)
    if (H.dims[i] < 1 || H.dims[i] > (1ull << 40)) return PC_ERR_CORRUPT;
  if (!make_geo(H.dims, H.block, g) || !shape_supported(H.block)) return PC_ERR_CORRUPT;
  if ((unsigned long long)g.nblocks != H.nblocks) return PC_ERR_CORRUPT;
  if (H.n_used > (1u << H.m)) return PC_ERR_CORRUPT;
  if (H.pred == 1) {
    if ((H.stencil != 7 && H.stencil != 13) || H.h1 < 2 || H.h1 > kMaxH || H.h2 < 0 || H.h2 > kMaxH ||
        H.s_in < 0 || H.s_in > 30 || H.nw != nweights(H.stencil, H.h1, H.h2) || H.nw > kMaxW)
      return PC_ERR_CORRUPT;
  } else if (H.pred == 2) {
    if (!qshape_ok(H.stencil, H.h1, H.h2) || H.s_in < 0 || H.s_in > 30 || H.nw != qnet_len(H.stencil, H.h1, H.h2))
      return PC_ERR_CORRUPT;
  } else if (H.pred != 0 || H.nw != 0) {
    return PC_ERR_CORRUPT;
  }
  const unsigned long long npts = (unsigned long long)H.dims[0] * H.dims[1] * H.dims[2];
  // every block stores its anchor as its first balance point
  if (H.n_out > npts || H.n_out < H.nblocks || H.swords > (npts * kLmax + 31) / 32 + 1) return PC_ERR_CORRUPT;
  const unsigned long long ts = H.dtype == PC_F64 ? 8 : 4;
  const unsigned long long ocb = al16(kHdr + (H.pred == 2 ? 8ull : 4ull) * H.nw);
  const unsigned long long obb = al16(ocb + 4ull * H.n_used);
  const unsigned long long obn = al16(obb + 4ull * H.nblocks);
  // balance values then stream, or (single pass) stream then balance values
  const bool sfirst = (flags & kFlagStreamFirst) != 0;
  const unsigned long long oov =
      sfirst ? al16(al16(obn + 2ull * H.nblocks) + 4ull * H.swords) : al16(obn + 2ull * H.nblocks);
  const unsigned long long ost = sfirst ? al16(obn + 2ull * H.nblocks) : al16(oov + ts * H.n_out);
  const unsigned long long tot = sfirst ? al16(oov + ts * H.n_out)
                                        : al16(ost + (H.lossless ? H.lzb : 4ull * H.swords));
  // the lossless section holds at most the stream and its chunk table
  if (H.lossless && H.lzb > al16(16 + 4 * lz_chunks_max(4ull * H.swords)) + 4ull * H.swords) return PC_ERR_CORRUPT;
  if (H.off_cb != ocb || H.off_bb != obb || H.off_bn != obn || H.off_ov != oov || H.off_st != ost || H.total != tot)
    return PC_ERR_CORRUPT;
  return PC_OK;
}

struct TrainLayout {
  size_t st, tabs, hist, cnt_t, cnt_v, off_t, off_v, tin, ttg, tus, vin, vtg, vus, w, lrs, lams, costs, ctl, qnet, qmax,
      shists, sbits, sst, slist, skey, sw, sparent, sdepth, sla, slb, srstart, ssymord, total;
  unsigned long long cap_t, cap_v;
};

bool train_shape_ok(int k, int h1, int h2) {
  return (k == 7 && h1 == 16 && h2 == 16) || (k == 13 && h1 == 32 && h2 == 32) || (k == 7 && h1 == 8 && h2 == 8) ||
         (k == 7 && h1 == 2 && h2 == 0) || (k == 13 && h1 == 16 && h2 == 16);
}

// Sample counts are drawn by a hash, so the buffers hold the expected count
// plus eight standard deviations (a larger draw is reported, not written).
TrainLayout train_layout(const Geo& g, int m, int k, int nw, unsigned int thr32, int nmodels) {
  const double p = (double)thr32 / 4294967296.0;
  const double n = (double)(g.n[0] * g.n[1] * g.n[2] - g.nblocks);
  const double mt = n * p * 0.8, mv = n * p * 0.2;
  TrainLayout L;
  L.cap_t = (unsigned long long)(mt + 8.0 * sqrt(mt + 1.0) + 256.0);
  L.cap_v = (unsigned long long)(mv + 8.0 * sqrt(mv + 1.0) + 256.0);
  const size_t nsym = (size_t)1 << m;
  size_t o = 0;
  L.st = o; o = up(o + sizeof(State));
  L.tabs = o; o = up(o + sizeof(Tabs));
  L.hist = o; o = up(o + 8 * nsym);
  L.cnt_t = o; o = up(o + 4 * (size_t)g.nblocks);
  L.cnt_v = o; o = up(o + 4 * (size_t)g.nblocks);
  L.off_t = o; o = up(o + 8 * (size_t)g.nblocks);
  L.off_v = o; o = up(o + 8 * (size_t)g.nblocks);
  L.tin = o; o = up(o + 4 * (size_t)k * L.cap_t);
  L.ttg = o; o = up(o + 4 * (size_t)L.cap_t);
  L.tus = o; o = up(o + (size_t)L.cap_t);
  L.vin = o; o = up(o + 4 * (size_t)k * L.cap_v);
  L.vtg = o; o = up(o + 4 * (size_t)L.cap_v);
  L.vus = o; o = up(o + (size_t)L.cap_v);
  L.w = o; o = up(o + 4 * (size_t)nw * nmodels);
  L.lrs = o; o = up(o + 4 * (size_t)nmodels);
  L.lams = o; o = up(o + 4 * (size_t)nmodels);
  L.costs = o; o = up(o + 8 * (size_t)(nmodels + 1));
  L.ctl = o; o = up(o + train_ctl_bytes());
  L.qnet = o; o = up(o + 8 * (size_t)qnet_len(13, 32, 32));
  L.qmax = o; o = up(o + 16);
  // selection by simulated compression (pc_train_select)
  size_t np = 1;
  while (np < nsym) np <<= 1;
  L.shists = o; o = up(o + 8 * nsym * (size_t)(nmodels + 1));
  L.sbits = o; o = up(o + 8 * 34 * (size_t)(nmodels + 1));
  L.sst = o; o = up(o + sizeof(State));
  L.slist = o; o = up(o + 4 * nsym + 64);
  L.skey = o; o = up(o + 8 * np);
  L.sw = o; o = up(o + 8 * 2 * nsym);
  L.sparent = o; o = up(o + 4 * 2 * nsym);
  L.sdepth = o; o = up(o + 4 * 2 * nsym);
  L.sla = o; o = up(o + 4 * nsym);
  L.slb = o; o = up(o + 4 * nsym);
  L.srstart = o; o = up(o + 4 * (nsym + 2));
  L.ssymord = o; o = up(o + 4 * nsym);
  L.total = o;
  return L;
}

TrainBufs train_bufs(const TrainLayout& L, uint8_t* ws) {
  TrainBufs tb;
  tb.cnt_t = reinterpret_cast<unsigned int*>(ws + L.cnt_t);
  tb.cnt_v = reinterpret_cast<unsigned int*>(ws + L.cnt_v);
  tb.off_t = reinterpret_cast<unsigned long long*>(ws + L.off_t);
  tb.off_v = reinterpret_cast<unsigned long long*>(ws + L.off_v);
  tb.tin = reinterpret_cast<int*>(ws + L.tin);
  tb.ttg = reinterpret_cast<int*>(ws + L.ttg);
  tb.tus = ws + L.tus;
  tb.vin = reinterpret_cast<int*>(ws + L.vin);
  tb.vtg = reinterpret_cast<int*>(ws + L.vtg);
  tb.vus = ws + L.vus;
  tb.w = reinterpret_cast<float*>(ws + L.w);
  tb.lrs = reinterpret_cast<const float*>(ws + L.lrs);
  tb.lams = reinterpret_cast<const float*>(ws + L.lams);
  tb.costs = reinterpret_cast<unsigned long long*>(ws + L.costs);
  tb.ctl = ws + L.ctl;
  tb.cap_t = L.cap_t;
  tb.cap_v = L.cap_v;
  return tb;
}

SelectBufs select_bufs(const TrainLayout& L, uint8_t* ws) {
  SelectBufs sb;
  sb.hists = reinterpret_cast<unsigned long long*>(ws + L.shists);
  sb.bitcnt = reinterpret_cast<unsigned long long*>(ws + L.sbits);
  sb.st = reinterpret_cast<State*>(ws + L.sst);
  sb.list = ws + L.slist;
  sb.hs.key = reinterpret_cast<unsigned long long*>(ws + L.skey);
  sb.hs.w = reinterpret_cast<unsigned long long*>(ws + L.sw);
  sb.hs.parent = reinterpret_cast<int*>(ws + L.sparent);
  sb.hs.depth = reinterpret_cast<int*>(ws + L.sdepth);
  sb.hs.la = reinterpret_cast<int*>(ws + L.sla);
  sb.hs.lb = reinterpret_cast<int*>(ws + L.slb);
  sb.hs.rstart = reinterpret_cast<int*>(ws + L.srstart);
  sb.hs.symord = reinterpret_cast<unsigned int*>(ws + L.ssymord);
  return sb;
}

// The coverage rule (Section IV.C) on residual bit-length counts cnt[0..33]:
// coverage(m) = share with bitlen <= m - 1; closest to 50% (eb < 1.5%) or 80%,
// the larger m on a tie.
int coverage_m(const unsigned long long* cnt, double eb) {
  unsigned long long used = 0;
  for (int b = 0; b < 34; ++b) used += cnt[b];
  if (used == 0) return 16;
  const double target = eb < 0.015 ? 0.5 : 0.8;
  int best = 16;
  double bestd = 2.0;
  for (int mm = 16; mm >= 2; --mm) {
    unsigned long long cov = 0;
    for (int b = 0; b <= mm - 1; ++b) cov += cnt[b];
    const double dd = fabs((double)cov / (double)used - target);
    if (dd < bestd) {
      bestd = dd;
      best = mm;
    }
  }
  return best;
}

int train_check(const size_t dims[3], int dtype, const pc_params* p, int nmodels, Geo& g, int& nw) {
  if (!dims || !p) return PC_ERR_ARG;
  if (dtype != PC_F32 && dtype != PC_F64) return PC_ERR_DTYPE;
  if (!(p->eb_rel > 0.0 && p->eb_rel < 1.0) || p->m < 2 || p->m > 16) return PC_ERR_ARG;
  if (!make_geo(dims, p->block, g) || nmodels < 1 || nmodels > 64) return PC_ERR_ARG;
  if (!train_shape_ok(p->stencil, p->hidden[0], p->hidden[1])) return PC_ERR_ARG;
  nw = nweights(p->stencil, p->hidden[0], p->hidden[1]);
  return PC_OK;
}

// Sampling threshold (of 2^32) of the training phase run inside pc_compress:
// p->train_samples expected non-anchor samples, or 10% of them.
unsigned int train_thr32(const size_t dims[3], const Geo& g, const pc_params* p) {
  const double n = (double)dims[0] * (double)dims[1] * (double)dims[2] - (double)g.nblocks;
  if (p->train_samples <= 0 || n <= 0.0) return (unsigned int)(0.1 * 4294967296.0);
  const double t = (double)p->train_samples / n * 4294967296.0;
  return t >= 4294967295.0 ? 4294967295u : (unsigned int)(t < 1.0 ? 1.0 : t);
}

// The library's (learning rate, L2 weight) grid of the training phase run
// inside pc_compress (Section IV.C trains several settings and keeps the best;
// the paper gives no values).
constexpr int kTrainModels = 16;
const float kGridLr[4] = {3e-3f, 1e-2f, 3e-2f, 1e-1f};
const float kGridLam[4] = {0.0f, 1e-5f, 1e-4f, 1e-3f};

// Everything one field's compression needs: layout of its workspace,
// header values, device pointers.
struct FieldPlan {
  const void* x;
  size_t dims[3];
  int dtype, mode, nw, m;
  double eb;
  Geo g;
  CompLayout L;
  HdrInfo hi;
  uint8_t* ws;
  uint8_t* out;
  State* stp;
  Tabs* tabs;
  unsigned long long* hist;
  uint16_t* codes;
  uint8_t* nnflag;
  uint32_t* nout;
  uint8_t* lens;
  uint32_t* cw;
  HuffScratch hs;
  const long long* h_qnet;  // host network to copy into the container (fixed-point form)
  const long long* qnet;    // its device copy in the container's weights section
  int literal, eq_period;  // the paper-literal selection
  LzBufs lz;               // the lossless stage (nch_max 0: off)
  // single pass (a given codebook)
  bool sp;
  const unsigned int* h_cb;
  int cb_n;
  unsigned long long off_bb, off_bn, off_st;
  unsigned long long* rec;
  uint32_t* side;
  unsigned long long* next;
  void* ov;
};

// Lay out one field's compression (checked parameters, explicit weights).
int plan_field(FieldPlan& F, const void* d_field, const size_t dims[3], int dtype, const pc_params* p, const Geo& g,
               int mode, int nw, void* d_out, size_t out_cap, void* d_ws, size_t ws_bytes, Mlp& mlp) {
  F.x = d_field;
  for (int i = 0; i < 3; ++i) F.dims[i] = dims[i];
  F.dtype = dtype;
  F.mode = mode;
  F.nw = nw;
  F.m = p->m;
  F.eb = p->eb_rel;
  F.g = g;
  F.L = comp_layout(g, p->m, p->h_codebook != nullptr, dtype == PC_F64 ? 8 : 4, p->lossless != 0);
  if (ws_bytes < F.L.total) return PC_ERR_CAPACITY;
  HdrInfo& hi = F.hi;
  hi.dtype = dtype;
  hi.pred = mode;
  hi.stencil = p->stencil;
  hi.h1 = p->hidden[0];
  hi.h2 = p->hidden[1];
  hi.m = p->m;
  hi.s_in = p->s_in;
  hi.nw = nw;
  hi.wsz = mode == 2 ? 8 : 4;
  hi.flags = (p->h_codebook ? kFlagStreamFirst : 0u) | (p->literal ? kFlagLiteral : 0u);
  hi.eq_period = p->literal ? p->eq_period : 0;
  hi.eb = p->eb_rel;
  hi.off_cb = al16(kHdr + (unsigned long long)hi.wsz * nw);
  hi.cap = out_cap;
  if (out_cap < hi.off_cb + 16) return PC_ERR_CAPACITY;
  memset(&mlp, 0, sizeof(Mlp));
  if (mode) {
    mlp.k = p->stencil;
    mlp.h1 = p->hidden[0];
    mlp.h2 = p->hidden[1];
    mlp.s_in = p->s_in;
    if (mode == 1) memcpy(mlp.w, p->h_weights, sizeof(float) * (size_t)nw);
  }
  const CompLayout& L = F.L;
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  F.ws = ws;
  F.out = static_cast<uint8_t*>(d_out);
  F.stp = reinterpret_cast<State*>(ws + L.st);
  F.tabs = reinterpret_cast<Tabs*>(ws + L.tabs);
  F.hist = reinterpret_cast<unsigned long long*>(ws + L.hist);
  F.codes = reinterpret_cast<uint16_t*>(ws + L.codes);
  F.nnflag = reinterpret_cast<uint8_t*>(ws + L.nnflag);
  F.nout = reinterpret_cast<uint32_t*>(ws + L.nout);
  F.lens = reinterpret_cast<uint8_t*>(ws + L.lens);
  F.cw = reinterpret_cast<uint32_t*>(ws + L.cw);
  F.hs.key = reinterpret_cast<unsigned long long*>(ws + L.key);
  F.hs.w = reinterpret_cast<unsigned long long*>(ws + L.w);
  F.hs.parent = reinterpret_cast<int*>(ws + L.parent);
  F.hs.depth = reinterpret_cast<int*>(ws + L.depth);
  F.hs.la = reinterpret_cast<int*>(ws + L.la);
  F.hs.lb = reinterpret_cast<int*>(ws + L.lb);
  F.hs.rstart = reinterpret_cast<int*>(ws + L.rstart);
  F.hs.symord = reinterpret_cast<unsigned int*>(ws + L.symord);
  // the fixed-point network goes straight into the container's weights
  // section, where the kernels read it
  F.h_qnet = mode == 2 ? p->h_qnet : nullptr;
  F.qnet = mode == 2 ? reinterpret_cast<const long long*>(F.out + kHdr) : nullptr;
  F.lz.nch_max = L.lz_nch;
  F.lz.slots = ws + L.lzslot;
  F.lz.sizes = reinterpret_cast<unsigned int*>(ws + L.lzsize);
  F.lz.offs = reinterpret_cast<unsigned long long*>(ws + L.lzoff);
  F.literal = p->literal;
  F.eq_period = p->eq_period;
  F.sp = p->h_codebook != nullptr;
  F.h_cb = p->h_codebook;
  F.cb_n = p->codebook_n;
  F.off_bb = al16(hi.off_cb + 4ull * (unsigned long long)(F.sp ? p->codebook_n : 0));
  F.off_bn = al16(F.off_bb + 4ull * (unsigned long long)g.nblocks);
  F.off_st = al16(F.off_bn + 2ull * (unsigned long long)g.nblocks);
  F.rec = reinterpret_cast<unsigned long long*>(ws + L.rec);
  F.side = reinterpret_cast<uint32_t*>(ws + L.side);
  F.next = reinterpret_cast<unsigned long long*>(ws + L.next);
  F.ov = ws + L.ov;
  if (F.sp && out_cap < F.off_st) return PC_ERR_CAPACITY;
  return PC_OK;
}

// a1, a2 (and the network into the container)
int launch_head(const FieldPlan& F, cudaStream_t s, int nsm) {
  if (F.mode == 2 &&
      cudaMemcpyAsync(F.out + kHdr, F.h_qnet, 8ull * F.nw, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PC_ERR_CUDA;
  const unsigned long long n = (unsigned long long)F.dims[0] * F.dims[1] * F.dims[2];
  const int nsym = 1 << F.m;
  int r = F.dtype == PC_F32 ? launch_stats_consts<float>(F.x, n, F.stp, F.tabs, F.hist, nsym, F.eb, nsm, s)
                            : launch_stats_consts<double>(F.x, n, F.stp, F.tabs, F.hist, nsym, F.eb, nsm, s);
  if (r || !F.sp) return r;
  // single pass: the codebook into the container and its code table, cleared
  // look-back records and brick counter
  const size_t nbk = (size_t)bricks_of(F.g);
  if (cudaMemcpyAsync(F.out + F.hi.off_cb, F.h_cb, 4ull * F.cb_n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(F.rec, 0, 16 * nbk, s) != cudaSuccess || cudaMemsetAsync(F.next, 0, 16, s) != cudaSuccess)
    return PC_ERR_CUDA;
  return launch_cb_table(F.out, F.hi.off_cb, F.cb_n, F.m, F.cw, F.stp, F.g, F.hi.cap, s);
}

CJob job_of(const FieldPlan& F) {
  CJob job{};
  job.x = F.x;
  job.g = F.g;
  job.st = F.stp;
  job.tabs = F.tabs;
  job.codes = F.codes;
  job.nnflag = F.nnflag;
  job.nout = F.nout;
  job.hist = F.hist;
  job.qnet = F.qnet;
  job.m = F.m;
  if (F.sp) {
    job.out = F.out;
    job.cwl = F.cw;
    job.rec = F.rec;
    job.side = F.side;
    job.ov = F.ov;
    job.off_bb = F.off_bb;
    job.off_bn = F.off_bn;
    job.off_st = F.off_st;
    job.cap_words = F.hi.cap > F.off_st ? (F.hi.cap - F.off_st) / 4 : 0;
    job.nbk = bricks_of(F.g);
  }
  return job;
}

// a10-a12 (single pass: only the finish)
int launch_tail(FieldPlan& F, const Mlp& mlp, cudaStream_t s, int nsm) {
  if (F.sp) {
    SpFinish f;
    f.rec = F.rec;
    f.side = F.side;
    f.ov = F.ov;
    f.nbk = bricks_of(F.g);
    f.off_bb = F.off_bb;
    f.off_bn = F.off_bn;
    f.off_st = F.off_st;
    return F.dtype == PC_F32 ? launch_sp_finish<float>(F.g, F.stp, F.out, F.hi, mlp, f, nsm, s)
                             : launch_sp_finish<double>(F.g, F.stp, F.out, F.hi, mlp, f, nsm, s);
  }
  int r = launch_codebook(F.hist, F.m, F.lens, F.cw, F.stp, F.hs, F.out, F.g, F.hi, s);
  if (r) return r;
  const CompLayout& L = F.L;
  auto* bbits = reinterpret_cast<uint32_t*>(F.ws + L.bbits);
  auto* cb = reinterpret_cast<unsigned long long*>(F.ws + L.cbits);
  auto* cn = reinterpret_cast<unsigned long long*>(F.ws + L.cnout);
  auto* cbo = reinterpret_cast<unsigned long long*>(F.ws + L.cboff);
  auto* coo = reinterpret_cast<unsigned long long*>(F.ws + L.cooff);
  r = F.dtype == PC_F32
          ? launch_pack<float>(static_cast<const float*>(F.x), F.g, F.codes, F.nnflag, F.nout, F.lens, F.cw, bbits, cb,
                               cn, cbo, coo, F.stp, F.out, F.hi, mlp, s)
          : launch_pack<double>(static_cast<const double*>(F.x), F.g, F.codes, F.nnflag, F.nout, F.lens, F.cw, bbits,
                                cb, cn, cbo, coo, F.stp, F.out, F.hi, mlp, s);
  if (r || F.lz.nch_max == 0) return r;
  return launch_lz_encode(F.out, F.hi.cap, F.stp, F.lz, s);
}

// Everything one container's decompression needs.
struct DecPlan {
  Hdr H;
  Geo g;
  DecLayout L;
  DecScratch ds;
  DecInfo di;
  const uint8_t* in;
  void* out;
  uint8_t* lzraw;                // the lossless stage's raw stream and chunk offsets (workspace)
  unsigned long long* lzoff;
};

// Parse and check a container (hbuf: its first `pre` host bytes) and lay out
// the decompression; fills the FP32 weights into mlp.
int plan_dec(DecPlan& P, const uint8_t* hbuf, size_t pre, const void* d_in, size_t in_size, void* d_field,
             size_t field_cap, void* d_ws, size_t ws_bytes, Mlp& mlp) {
  Hdr& H = P.H;
  int st = parse_header(hbuf, pre, H, P.g);
  if (st) return st;
  if (H.total > in_size) return PC_ERR_CORRUPT;
  const size_t ts = H.dtype == PC_F64 ? 8 : 4;
  const size_t n = H.dims[0] * H.dims[1] * H.dims[2];
  if (field_cap < n * ts) return PC_ERR_CAPACITY;
  P.L = dec_layout(P.g, H.m, H.lossless ? 4ull * H.swords : 0ull);
  const DecLayout& L = P.L;
  if (ws_bytes < L.total) return PC_ERR_CAPACITY;
  memset(&mlp, 0, sizeof(Mlp));
  if (H.pred == 1 || H.pred == 2) {
    mlp.k = H.stencil;
    mlp.h1 = H.h1;
    mlp.h2 = H.h2;
    mlp.s_in = H.s_in;
  }
  if (H.pred == 1) {
    // nw <= kMaxW (checked with the header) and the container holds the section
    if (kHdr + 4ull * H.nw > pre) return PC_ERR_CORRUPT;
    memcpy(mlp.w, hbuf + kHdr, 4ull * H.nw);
  }
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  DecScratch& ds = P.ds;
  ds.err = reinterpret_cast<int*>(ws + L.err);
  ds.ftab = reinterpret_cast<Tabs*>(ws + L.ftab);
  ds.sorted = reinterpret_cast<uint16_t*>(ws + L.sorted);
  ds.tabs = reinterpret_cast<unsigned int*>(ws + L.tabs);
  ds.chunk_bits = reinterpret_cast<unsigned long long*>(ws + L.cbits);
  ds.chunk_nout = reinterpret_cast<unsigned long long*>(ws + L.cnout);
  ds.chunk_boff = reinterpret_cast<unsigned long long*>(ws + L.cboff);
  ds.chunk_ooff = reinterpret_cast<unsigned long long*>(ws + L.cooff);
  ds.boff = reinterpret_cast<unsigned long long*>(ws + L.boff);
  ds.ooff = reinterpret_cast<unsigned long long*>(ws + L.ooff);
  ds.codes = reinterpret_cast<uint16_t*>(ws + L.codes);
  DecInfo& di = P.di;
  di.dtype = H.dtype;
  di.m = H.m;
  di.stencil = H.pred != 0 ? H.stencil : 7;
  di.h1 = H.h1;
  di.h2 = H.h2;
  di.s_in = H.s_in;
  di.usenn_any = H.pred != 0;
  di.qmode = H.pred == 2;
  di.literal = H.literal;
  // the fixed-point network is read in place from the container
  di.qnet = H.pred == 2 ? reinterpret_cast<const long long*>(static_cast<const uint8_t*>(d_in) + kHdr) : nullptr;
  di.n_used = H.n_used;
  di.n_out = H.n_out;
  di.swords = H.swords;
  di.off_cb = H.off_cb;
  di.off_bb = H.off_bb;
  di.off_bn = H.off_bn;
  di.off_ov = H.off_ov;
  di.off_st = H.off_st;
  // the bitstream: in place, or the lossless stage's output in the workspace
  P.lzraw = ws + L.lzraw;
  P.lzoff = reinterpret_cast<unsigned long long*>(ws + L.lzoff);
  di.stream = H.lossless ? P.lzraw : static_cast<const uint8_t*>(d_in) + H.off_st;
  di.in_size = in_size;
  di.Kp = H.Kp;
  di.Kn = H.Kn;
  di.Zq = H.Zq;
  di.S = H.S;
  di.step_bits = H.step_bits;
  di.inv_bits = H.inv_bits;
  di.ebdn_bits = H.ebdn_bits;
  P.in = static_cast<const uint8_t*>(d_in);
  P.out = d_field;
  return PC_OK;
}

int launch_dec(const DecPlan& P, const Mlp& mlp, int nsm, cudaStream_t s, SlabSink* sink = nullptr,
               int phase = kDecAll) {
  if (phase != kDecRecon && cudaMemsetAsync(P.ds.err, 0, sizeof(int), s) != cudaSuccess) return PC_ERR_CUDA;
  if (phase != kDecRecon && P.H.lossless) {
    // the fourth SZ stage undone first: the raw words (and zero padding) for the Huffman decoder
    const unsigned long long nraw = 4ull * P.H.swords;
    if (cudaMemsetAsync(P.lzraw + nraw, 0, al16(nraw) + 64 - nraw, s) != cudaSuccess) return PC_ERR_CUDA;
    const int r = launch_lz_decode(P.in + P.H.off_st, P.H.lzb, nraw, P.lzraw, P.lzoff, P.ds.err, s);
    if (r) return r;
  }
  return P.H.dtype == PC_F32
             ? launch_decompress<float>(P.in, P.g, P.di, P.ds, mlp, static_cast<float*>(P.out), nsm, s, sink, phase)
             : launch_decompress<double>(P.in, P.g, P.di, P.ds, mlp, static_cast<double*>(P.out), nsm, s, sink,
                                         phase);
}

// Streams of the batched decoder's reconstructions (and their fork and join
// events), one set per host thread and device, created on first use and kept.
constexpr int kAuxStreams = 4;
struct AuxStreams {
  cudaStream_t s[kAuxStreams];
  cudaEvent_t fork, join[kAuxStreams];
};
AuxStreams* aux_streams() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  static thread_local AuxStreams sets[64];
  static thread_local bool ready[64];
  AuxStreams& a = sets[dev];
  if (!ready[dev]) {
    for (int i = 0; i < kAuxStreams; ++i)
      if (cudaStreamCreateWithFlags(&a.s[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&a.join[i], cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    if (cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    ready[dev] = true;
  }
  return &a;
}

// Work recorded on s so far runs before anything later on the aux streams.
int aux_fork(AuxStreams* a, cudaStream_t s) {
  if (!a || cudaEventRecord(a->fork, s) != cudaSuccess) return PC_ERR_CUDA;
  for (int i = 0; i < kAuxStreams; ++i)
    if (cudaStreamWaitEvent(a->s[i], a->fork, 0) != cudaSuccess) return PC_ERR_CUDA;
  return PC_OK;
}

// Everything recorded on the aux streams so far runs before anything later on s.
int aux_join(AuxStreams* a, cudaStream_t s) {
  for (int i = 0; i < kAuxStreams; ++i)
    if (cudaEventRecord(a->join[i], a->s[i]) != cudaSuccess || cudaStreamWaitEvent(s, a->join[i], 0) != cudaSuccess)
      return PC_ERR_CUDA;
  return PC_OK;
}

// The copy stream and events of the host-buffer decoder, one set per host
// thread and device, created on first use and kept for the thread's life.
SlabSink* host_sink(void* h_field) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  static thread_local SlabSink sinks[64];
  static thread_local bool ready[64];
  SlabSink& k = sinks[dev];
  if (!ready[dev]) {
    if (cudaStreamCreateWithFlags(&k.cs, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    for (int i = 0; i <= kSlabs; ++i)
      if (cudaEventCreateWithFlags(&k.ev[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    ready[dev] = true;
  }
  k.host = h_field;
  k.used = false;
  return &k;
}

}  // namespace

extern "C" {

int pc_train_workspace_size(const size_t dims[3], int dtype, const pc_params* p, unsigned int thr32, int nmodels,
                            size_t* ws_bytes) {
  Geo g;
  int nw;
  int st = train_check(dims, dtype, p, nmodels, g, nw);
  if (st) return st;
  if (!ws_bytes) return PC_ERR_ARG;
  *ws_bytes = train_layout(g, p->m, p->stencil, nw, thr32, nmodels).total;
  return PC_OK;
}

}  // extern "C"

namespace {

// The training phase; with select, the models are scored by simulated
// compression and m comes from the coverage rule (pc_train_select).
int train_run(const void* d_field, const size_t dims[3], int dtype, const pc_params* p, unsigned long long seed,
              unsigned int thr32, int nmodels, const float* h_lrs, const float* h_lams, float* h_weights_out,
              int* s_in_out, int* chosen_out, unsigned long long* h_costs, bool select, int* m_out, void* d_ws,
              size_t ws_bytes, void* stream) {
  Geo g;
  int nw;
  int st = train_check(dims, dtype, p, nmodels, g, nw);
  if (st) return st;
  if (!d_field || !h_lrs || !h_lams || !h_weights_out || !s_in_out || !chosen_out || !d_ws) return PC_ERR_ARG;
  TrainLayout L = train_layout(g, p->m, p->stencil, nw, thr32, nmodels);
  if (ws_bytes < L.total) return PC_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nsm = sm_count();
  if (nsm <= 0) return PC_ERR_CUDA;
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  State* stp = reinterpret_cast<State*>(ws + L.st);
  Tabs* tabs = reinterpret_cast<Tabs*>(ws + L.tabs);
  auto* hist = reinterpret_cast<unsigned long long*>(ws + L.hist);
  TrainBufs tb = train_bufs(L, ws);
  if (cudaMemcpyAsync(ws + L.lrs, h_lrs, 4ull * nmodels, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(ws + L.lams, h_lams, 4ull * nmodels, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PC_ERR_CUDA;
  const unsigned long long n = (unsigned long long)dims[0] * dims[1] * dims[2];
  const int nsym = 1 << p->m;
  int r;
  if (dtype == PC_F32) {
    r = launch_stats_consts<float>(d_field, n, stp, tabs, hist, nsym, p->eb_rel, nsm, s);
    if (!r) r = launch_train<float>(static_cast<const float*>(d_field), g, stp, tabs, tb, p->stencil, p->hidden[0],
                                   p->hidden[1], p->m, nmodels, seed, thr32, s);
  } else {
    r = launch_stats_consts<double>(d_field, n, stp, tabs, hist, nsym, p->eb_rel, nsm, s);
    if (!r) r = launch_train<double>(static_cast<const double*>(d_field), g, stp, tabs, tb, p->stencil, p->hidden[0],
                                    p->hidden[1], p->m, nmodels, seed, thr32, s);
  }
  SelectBufs sb = select_bufs(L, ws);
  if (!r && select)
    r = launch_select(tb, sb, p->stencil, p->hidden[0], p->hidden[1], p->m, nmodels, dtype == PC_F64 ? 64 : 32, s);
  if (r) return r;
  unsigned long long ctl[8];
  int herr = 0;
  if (cudaMemcpyAsync(ctl, tb.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&herr, &stp->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(h_weights_out, tb.w, 4ull * nw * nmodels, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PC_ERR_CUDA;
  unsigned long long costs[65];
  if (cudaMemcpyAsync(costs, tb.costs, 8ull * (nmodels + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PC_ERR_CUDA;
  static thread_local unsigned long long bitcnt[65 * 34];
  if (select && cudaMemcpyAsync(bitcnt, sb.bitcnt, 8ull * 34 * (nmodels + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  prof_collect();
  if (herr) return herr;
  // TrainCtl: ntrain, nval, s2, nused, then {s_in, chosen, err, pad}
  if (ctl[0] > L.cap_t || ctl[1] > L.cap_v) return PC_ERR_CAPACITY;
  int tail[4];
  memcpy(tail, &ctl[4], sizeof(tail));
  *s_in_out = tail[0];
  *chosen_out = tail[1];
  if (h_costs) memcpy(h_costs, costs, 8ull * (nmodels + 1));
  if (select && m_out) {
    const int c = tail[1] >= 0 ? tail[1] : nmodels;
    *m_out = coverage_m(bitcnt + 34 * c, p->eb_rel);
  }
  return PC_OK;
}

}  // namespace

extern "C" {

int pc_train(const void* d_field, const size_t dims[3], int dtype, const pc_params* p, unsigned long long seed,
             unsigned int thr32, int nmodels, const float* h_lrs, const float* h_lams, float* h_weights_out,
             int* s_in_out, int* chosen_out, unsigned long long* h_costs, void* d_ws, size_t ws_bytes,
             void* stream) {
  return train_run(d_field, dims, dtype, p, seed, thr32, nmodels, h_lrs, h_lams, h_weights_out, s_in_out, chosen_out,
                   h_costs, false, nullptr, d_ws, ws_bytes, stream);
}

int pc_train_select(const void* d_field, const size_t dims[3], int dtype, const pc_params* p,
                    unsigned long long seed, unsigned int thr32, int nmodels, const float* h_lrs,
                    const float* h_lams, float* h_weights_out, int* s_in_out, int* chosen_out,
                    unsigned long long* h_sizes, int* m_out, void* d_ws, size_t ws_bytes, void* stream) {
  if (!m_out) return PC_ERR_ARG;
  return train_run(d_field, dims, dtype, p, seed, thr32, nmodels, h_lrs, h_lams, h_weights_out, s_in_out, chosen_out,
                   h_sizes, true, m_out, d_ws, ws_bytes, stream);
}

int pc_sample_codebook(const void* d_field, const size_t dims[3], int dtype, const pc_params* p,
                       unsigned long long seed, unsigned int thr32, int span_fill, unsigned int* h_codebook_out,
                       int* n_out, void* d_ws, size_t ws_bytes, void* stream) {
  if (!p || !d_field || !h_codebook_out || !n_out || !d_ws) return PC_ERR_ARG;
  const bool lorenzo = p->pred == PC_PRED_LORENZO;
  if (!lorenzo && (p->pred != PC_PRED_MLP_FP32 && p->pred != PC_PRED_MLP_BF16)) return PC_ERR_ARG;
  if (!lorenzo && (!p->h_weights || p->s_in < 0 || p->s_in > 30)) return PC_ERR_ARG;
  // the sampling and the histogram run on the training phase's buffers
  pc_params tp = *p;
  if (lorenzo) {
    tp.stencil = 7;
    tp.hidden[0] = 16;
    tp.hidden[1] = 16;
  }
  Geo g;
  int nw;
  int st = train_check(dims, dtype, &tp, 1, g, nw);
  if (st) return st;
  TrainLayout L = train_layout(g, tp.m, tp.stencil, nw, thr32, 1);
  if (ws_bytes < L.total) return PC_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nsm = sm_count();
  if (nsm <= 0) return PC_ERR_CUDA;
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  State* stp = reinterpret_cast<State*>(ws + L.st);
  Tabs* tabs = reinterpret_cast<Tabs*>(ws + L.tabs);
  auto* hist = reinterpret_cast<unsigned long long*>(ws + L.hist);
  TrainBufs tb = train_bufs(L, ws);
  SelectBufs sb = select_bufs(L, ws);
  if ((lorenzo ? cudaMemsetAsync(tb.w, 0, 4ull * nw, s)
               : cudaMemcpyAsync(tb.w, p->h_weights, 4ull * nw, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return PC_ERR_CUDA;
  const unsigned long long n = (unsigned long long)dims[0] * dims[1] * dims[2];
  const int nsym = 1 << tp.m;
  int r;
  if (dtype == PC_F32) {
    r = launch_stats_consts<float>(d_field, n, stp, tabs, hist, nsym, tp.eb_rel, nsm, s);
    if (!r) r = launch_sample_hist<float>(static_cast<const float*>(d_field), g, stp, tabs, tb, sb, tp.stencil,
                                         tp.hidden[0], tp.hidden[1], tp.s_in, tp.m, lorenzo, span_fill, seed, thr32, s);
  } else {
    r = launch_stats_consts<double>(d_field, n, stp, tabs, hist, nsym, tp.eb_rel, nsm, s);
    if (!r) r = launch_sample_hist<double>(static_cast<const double*>(d_field), g, stp, tabs, tb, sb, tp.stencil,
                                          tp.hidden[0], tp.hidden[1], tp.s_in, tp.m, lorenzo, span_fill, seed, thr32, s);
  }
  if (r) return r;
  unsigned long long ctl[8];
  int herr = 0;
  State hs;
  if (cudaMemcpyAsync(ctl, tb.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&herr, &stp->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&hs, sb.st, sizeof(State), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(h_codebook_out, sb.list, 4ull * nsym, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  prof_collect();
  if (herr) return herr;
  if (hs.err) return hs.err;
  if (ctl[0] > L.cap_t || ctl[1] > L.cap_v) return PC_ERR_CAPACITY;
  *n_out = (int)hs.n_used;
  return PC_OK;
}

int pc_quantize(const void* d_field, const size_t dims[3], int dtype, const pc_params* p, unsigned long long seed,
                unsigned int thr32, long long* h_qnet_out, void* d_ws, size_t ws_bytes, void* stream) {
  Geo g;
  int nw;
  int st = train_check(dims, dtype, p, 1, g, nw);
  if (st) return st;
  if (!d_field || !p->h_weights || !h_qnet_out || !d_ws || p->s_in < 0 || p->s_in > 30) return PC_ERR_ARG;
  if (!qshape_ok(p->stencil, p->hidden[0], p->hidden[1])) return PC_ERR_ARG;
  TrainLayout L = train_layout(g, p->m, p->stencil, nw, thr32, 1);
  if (ws_bytes < L.total) return PC_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nsm = sm_count();
  if (nsm <= 0) return PC_ERR_CUDA;
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  State* stp = reinterpret_cast<State*>(ws + L.st);
  Tabs* tabs = reinterpret_cast<Tabs*>(ws + L.tabs);
  auto* hist = reinterpret_cast<unsigned long long*>(ws + L.hist);
  TrainBufs tb;
  tb.cnt_t = reinterpret_cast<unsigned int*>(ws + L.cnt_t);
  tb.cnt_v = reinterpret_cast<unsigned int*>(ws + L.cnt_v);
  tb.off_t = reinterpret_cast<unsigned long long*>(ws + L.off_t);
  tb.off_v = reinterpret_cast<unsigned long long*>(ws + L.off_v);
  tb.tin = reinterpret_cast<int*>(ws + L.tin);
  tb.ttg = reinterpret_cast<int*>(ws + L.ttg);
  tb.tus = ws + L.tus;
  tb.vin = reinterpret_cast<int*>(ws + L.vin);
  tb.vtg = reinterpret_cast<int*>(ws + L.vtg);
  tb.vus = ws + L.vus;
  tb.w = reinterpret_cast<float*>(ws + L.w);
  tb.lrs = nullptr;
  tb.lams = nullptr;
  tb.costs = reinterpret_cast<unsigned long long*>(ws + L.costs);
  tb.ctl = ws + L.ctl;
  tb.cap_t = L.cap_t;
  tb.cap_v = L.cap_v;
  auto* q = reinterpret_cast<long long*>(ws + L.qnet);
  auto* qmax = reinterpret_cast<unsigned long long*>(ws + L.qmax);
  if (cudaMemcpyAsync(tb.w, p->h_weights, 4ull * nw, cudaMemcpyHostToDevice, s) != cudaSuccess) return PC_ERR_CUDA;
  const unsigned long long n = (unsigned long long)dims[0] * dims[1] * dims[2];
  const int nsym = 1 << p->m;
  int r;
  if (dtype == PC_F32) {
    r = launch_stats_consts<float>(d_field, n, stp, tabs, hist, nsym, p->eb_rel, nsm, s);
    if (!r) r = launch_quantize<float>(static_cast<const float*>(d_field), g, stp, tabs, tb, p->stencil, p->hidden[0],
                                      p->hidden[1], p->s_in, seed, thr32, q, qmax, s);
  } else {
    r = launch_stats_consts<double>(d_field, n, stp, tabs, hist, nsym, p->eb_rel, nsm, s);
    if (!r) r = launch_quantize<double>(static_cast<const double*>(d_field), g, stp, tabs, tb, p->stencil,
                                       p->hidden[0], p->hidden[1], p->s_in, seed, thr32, q, qmax, s);
  }
  if (r) return r;
  const int len = qnet_len(p->stencil, p->hidden[0], p->hidden[1]);
  unsigned long long ctl[8];
  int herr = 0;
  if (cudaMemcpyAsync(ctl, tb.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&herr, &stp->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(h_qnet_out, q, 8ull * len, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  if (herr) return herr;
  if (ctl[0] > L.cap_t || ctl[1] > L.cap_v) return PC_ERR_CAPACITY;
  return qnet_valid(h_qnet_out, p->stencil, p->hidden[0], p->hidden[1], p->s_in) ? PC_OK : PC_ERR_ARG;
}

int pc_qnet_len(int k, int h1, int h2) { return qnet_len(k, h1, h2); }

int pc_mlp_nweights(int k, int h1, int h2) { return nweights(k, h1, h2); }

size_t pc_compress_bound(const size_t dims[3], int dtype, const pc_params* p) {
  Geo g;
  int mode, nw;
  if (check_params(dims, dtype, p, g, mode, nw) != PC_OK) return 0;
  if (wants_training(p))  // the network chosen inside the call (or none)
    nw = mode == 2 ? qnet_len(p->stencil, p->hidden[0], p->hidden[1]) : nweights(p->stencil, p->hidden[0], p->hidden[1]);
  const unsigned long long n = (unsigned long long)dims[0] * dims[1] * dims[2];
  const unsigned long long ts = dtype == PC_F64 ? 8 : 4;
  unsigned long long b = kHdr;
  b = al16(b + (mode == 2 ? 8ull : 4ull) * nw);
  b = al16(b + 4ull * (1ull << p->m));
  b = al16(b + 4ull * g.nblocks);
  b = al16(b + 2ull * g.nblocks);
  b = al16(b + ts * n);
  b = al16(b + stream_bytes_max(n));
  // the lossless stage's section header and chunk table (a chunk is never stored longer than itself)
  if (p->lossless) b += al16(16 + 4 * lz_chunks_max(stream_bytes_max(n))) + 16;
  return (size_t)b;
}

int pc_compress_workspace_size(const size_t dims[3], int dtype, const pc_params* p, size_t* ws) {
  Geo g;
  int mode, nw;
  int st = check_params(dims, dtype, p, g, mode, nw);
  if (st) return st;
  if (!ws) return PC_ERR_ARG;
  *ws = comp_layout(g, p->m, p->h_codebook != nullptr, dtype == PC_F64 ? 8 : 4, p->lossless != 0).total;
  if (wants_training(p)) {
    const size_t tw = train_layout(g, p->m, p->stencil, nweights(p->stencil, p->hidden[0], p->hidden[1]),
                                   train_thr32(dims, g, p), kTrainModels).total;
    if (tw > *ws) *ws = tw;
  }
  return PC_OK;
}

int pc_compress_workspace_layout(const size_t dims[3], int dtype, const pc_params* p, size_t* off_codes,
                                 size_t* off_nnflag, size_t* off_hist) {
  Geo g;
  int mode, nw;
  int st = check_params(dims, dtype, p, g, mode, nw);
  if (st) return st;
  CompLayout L = comp_layout(g, p->m, p->h_codebook != nullptr, dtype == PC_F64 ? 8 : 4, p->lossless != 0);
  if (off_codes) *off_codes = L.codes;
  if (off_nnflag) *off_nnflag = L.nnflag;
  if (off_hist) *off_hist = L.hist;
  return PC_OK;
}

int pc_compress(const void* d_field, const size_t dims[3], int dtype, const pc_params* p, void* d_out,
                size_t out_cap, size_t* out_size, void* d_ws, size_t ws_bytes, void* stream) {
  Geo g;
  int mode, nw;
  int st = check_params(dims, dtype, p, g, mode, nw);
  if (st) return st;
  if (!d_field || !d_out || !out_size || !d_ws) return PC_ERR_ARG;
  if (wants_training(p)) {
    // the learned part on the device (Section IV.C), then compression with its choice
    size_t need = 0;
    st = pc_compress_workspace_size(dims, dtype, p, &need);
    if (st) return st;
    if (ws_bytes < need) return PC_ERR_CAPACITY;
    pc_params tp = *p;
    tp.pred = PC_PRED_MLP_FP32;
    tp.h_weights = nullptr;
    tp.h_qnet = nullptr;
    const int nwt = nweights(p->stencil, p->hidden[0], p->hidden[1]);
    static thread_local float W[kTrainModels * kMaxW];
    static thread_local long long Q[kQHdr + 2 * kMaxH * 13 + kMaxH * kMaxH + 4 * kMaxH + 1];
    float lrs[kTrainModels], lams[kTrainModels];
    for (int i = 0; i < kTrainModels; ++i) {
      lrs[i] = kGridLr[i / 4];
      lams[i] = kGridLam[i % 4];
    }
    const unsigned int thr32 = train_thr32(dims, g, p);
    int s_in = 0, chosen = -1;
    st = pc_train(d_field, dims, dtype, &tp, p->seed, thr32, kTrainModels, lrs, lams, W, &s_in, &chosen, nullptr,
                  d_ws, ws_bytes, stream);
    if (st) return st;
    pc_params cp = *p;
    if (chosen < 0) {
      cp.pred = PC_PRED_LORENZO;
    } else {
      cp.s_in = s_in;
      cp.h_weights = W + (size_t)chosen * nwt;
      if (mode == 2) {
        st = pc_quantize(d_field, dims, dtype, &cp, p->seed, thr32, Q, d_ws, ws_bytes, stream);
        if (st) return st;
        cp.h_qnet = Q;
      }
    }
    return pc_compress(d_field, dims, dtype, &cp, d_out, out_cap, out_size, d_ws, ws_bytes, stream);
  }
  static thread_local Mlp mlp;
  FieldPlan F;
  st = plan_field(F, d_field, dims, dtype, p, g, mode, nw, d_out, out_cap, d_ws, ws_bytes, mlp);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nsm = sm_count();
  if (nsm <= 0) return PC_ERR_CUDA;
  int r = launch_head(F, s, nsm);
  if (!r && F.literal) {
    r = launch_lit_compress(static_cast<const float*>(F.x), F.g, F.stp, F.tabs, mlp, mode, F.eq_period, F.m, F.codes,
                            F.nnflag, F.nout, F.hist, nsm, s);
  } else if (!r) {
    const CJob job = job_of(F);
    unsigned long long* next = F.sp ? F.next : nullptr;
    r = dtype == PC_F32 ? launch_compress<float>(&job, 1, mode, mlp, nsm, s, next)
                        : launch_compress<double>(&job, 1, mode, mlp, nsm, s, next);
  }
  if (!r) r = launch_tail(F, mlp, s, nsm);
  if (r) return r;
  State hst;
  if (cudaMemcpyAsync(&hst, F.stp, sizeof(State), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  prof_collect();
  if (hst.err) return hst.err;
  *out_size = (size_t)hst.out_size;
  return PC_OK;
}

int pc_compress_batch_workspace_size(int nfields, const size_t* dims, const int* dtypes, const pc_params* params,
                                     size_t* ws_bytes, size_t* out_bytes) {
  if (nfields < 1 || !dims || !dtypes || !params || !ws_bytes || !out_bytes) return PC_ERR_ARG;
  size_t ws = 0, ob = 0;
  for (int i = 0; i < nfields; ++i) {
    Geo g;
    int mode, nw;
    int st = check_params(dims + 3 * i, dtypes[i], params + i, g, mode, nw);
    if (st) return st;
    if (wants_training(params + i) || params[i].literal) return PC_ERR_ARG;
    ws += up(comp_layout(g, params[i].m, params[i].h_codebook != nullptr, dtypes[i] == PC_F64 ? 8 : 4, params[i].lossless != 0).total);
    ob += up(pc_compress_bound(dims + 3 * i, dtypes[i], params + i));
  }
  *ws_bytes = ws;
  *out_bytes = ob;
  return PC_OK;
}

int pc_compress_batch(int nfields, const void* const* d_fields, const size_t* dims, const int* dtypes,
                      const pc_params* params, void* d_out, size_t out_cap, size_t* offsets, size_t* sizes,
                      void* d_ws, size_t ws_bytes, void* stream) {
  if (nfields < 1 || !d_fields || !dims || !dtypes || !params || !d_out || !offsets || !sizes || !d_ws)
    return PC_ERR_ARG;
  size_t need_ws = 0, need_out = 0;
  int st = pc_compress_batch_workspace_size(nfields, dims, dtypes, params, &need_ws, &need_out);
  if (st) return st;
  if (ws_bytes < need_ws || out_cap < need_out) return PC_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nsm = sm_count();
  if (nsm <= 0) return PC_ERR_CUDA;
  std::vector<FieldPlan> F((size_t)nfields);
  std::vector<Mlp> mlps((size_t)nfields);
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  uint8_t* out = static_cast<uint8_t*>(d_out);
  size_t wo = 0, oo = 0;
  for (int i = 0; i < nfields; ++i) {
    Geo g;
    int mode, nw;
    check_params(dims + 3 * i, dtypes[i], params + i, g, mode, nw);
    const size_t wsz = up(comp_layout(g, params[i].m, params[i].h_codebook != nullptr, dtypes[i] == PC_F64 ? 8 : 4, params[i].lossless != 0).total);
    const size_t osz = up(pc_compress_bound(dims + 3 * i, dtypes[i], params + i));
    offsets[i] = oo;
    st = plan_field(F[i], d_fields[i], dims + 3 * i, dtypes[i], params + i, g, mode, nw, out + oo, osz, ws + wo, wsz,
                    mlps[i]);
    if (st) return st;
    wo += wsz;
    oo += osz;
  }
  offsets[nfields] = oo;
  // a1, a2 per field, on a few streams of their own so that small fields run side by side
  AuxStreams* aux = aux_streams();
  if ((st = aux_fork(aux, s))) return st;
  for (int i = 0; i < nfields; ++i)
    if ((st = launch_head(F[i], aux->s[i % kAuxStreams], nsm))) return st;
  if ((st = aux_join(aux, s))) return st;
  // a4-a9: one persistent launch per group of fields that share dtype, block
  // shape and predictor form (and, for the FP32 form, the weights)
  std::vector<int> done((size_t)nfields, 0);
  std::vector<CJob> jl;
  auto same_launch = [&](int i, int j) {
    const pc_params& pi = params[i];
    const pc_params& pj = params[j];
    return dtypes[j] == dtypes[i] && F[j].mode == F[i].mode && pj.block[0] == pi.block[0] &&
           pj.block[1] == pi.block[1] && pj.block[2] == pi.block[2] &&
           (F[i].mode == 0 ||
            (pj.stencil == pi.stencil && pj.hidden[0] == pi.hidden[0] && pj.hidden[1] == pi.hidden[1])) &&
           (F[i].mode != 1 || (pj.h_weights == pi.h_weights && pj.s_in == pi.s_in)) && F[j].sp == F[i].sp;
  };
  for (;;) {
    int i = 0;
    while (i < nfields && done[i]) ++i;
    if (i == nfields) break;
    jl.clear();
    for (int j = i; j < nfields && (int)jl.size() < kMaxJobs; ++j)
      if (!done[j] && same_launch(i, j)) {
        jl.push_back(job_of(F[j]));
        done[j] = 1;
      }
    unsigned long long* next = F[i].sp ? F[i].next : nullptr;
    st = dtypes[i] == PC_F32 ? launch_compress<float>(jl.data(), (int)jl.size(), F[i].mode, mlps[i], nsm, s, next)
                             : launch_compress<double>(jl.data(), (int)jl.size(), F[i].mode, mlps[i], nsm, s, next);
    if (st) return st;
  }
  // a10-a12 per field, on the aux streams again
  if ((st = aux_fork(aux, s))) return st;
  for (int i = 0; i < nfields; ++i)
    if ((st = launch_tail(F[i], mlps[i], aux->s[i % kAuxStreams], nsm))) return st;
  if ((st = aux_join(aux, s))) return st;
  std::vector<State> hs((size_t)nfields);
  for (int i = 0; i < nfields; ++i)
    if (cudaMemcpyAsync(&hs[i], F[i].stp, sizeof(State), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  prof_collect();
  int err = PC_OK;
  for (int i = 0; i < nfields; ++i) {
    if (hs[i].err && !err) err = hs[i].err;
    sizes[i] = (size_t)hs[i].out_size;
  }
  return err;
}

int pc_decompress_batch_workspace_size(int nfields, const void* const* h_headers, size_t* ws_bytes) {
  if (nfields < 1 || !h_headers || !ws_bytes) return PC_ERR_ARG;
  size_t ws = 0;
  for (int i = 0; i < nfields; ++i) {
    size_t w = 0;
    int st = pc_header_info(h_headers[i], kHdr, nullptr, nullptr, &w);
    if (st) return st;
    ws += up(w);
  }
  *ws_bytes = ws;
  return PC_OK;
}

int pc_decompress_batch(int nfields, const void* d_in, const size_t* offsets, const size_t* sizes,
                        void* const* d_fields, const size_t* field_caps, void* d_ws, size_t ws_bytes, void* stream) {
  if (nfields < 1 || !d_in || !offsets || !sizes || !d_fields || !field_caps || !d_ws) return PC_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint8_t* in = static_cast<const uint8_t*>(d_in);
  // every header (and FP32 weight section) in one read-back
  const size_t hb = kHdr + 4 * kMaxW;
  std::vector<uint8_t> hbuf((size_t)nfields * hb);
  std::vector<size_t> pre((size_t)nfields);
  for (int i = 0; i < nfields; ++i) {
    if (sizes[i] < (size_t)kHdr) return PC_ERR_CORRUPT;
    pre[i] = sizes[i] < hb ? sizes[i] : hb;
    if (cudaMemcpyAsync(hbuf.data() + (size_t)i * hb, in + offsets[i], pre[i], cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
      return PC_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  const int nsm = sm_count();
  if (nsm <= 0) return PC_ERR_CUDA;
  std::vector<DecPlan> P((size_t)nfields);
  std::vector<Mlp> mlps((size_t)nfields);
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  size_t wo = 0;
  for (int i = 0; i < nfields; ++i) {
    size_t w = 0;
    int st = pc_header_info(hbuf.data() + (size_t)i * hb, kHdr, nullptr, nullptr, &w);
    if (st) return st;
    w = up(w);
    if (wo + w > ws_bytes) return PC_ERR_CAPACITY;
    st = plan_dec(P[i], hbuf.data() + (size_t)i * hb, pre[i], in + offsets[i], sizes[i], d_fields[i], field_caps[i],
                  ws + wo, w, mlps[i]);
    if (st) return st;
    wo += w;
  }
  // tables and offsets per field, the Huffman decoders of up to 32 fields in one launch (small fields alone
  // fill few SMs), then each field's reconstruction
  for (int i = 0; i < nfields; ++i) {
    int st = launch_dec(P[i], mlps[i], nsm, s, nullptr, kDecPrep);
    if (st) return st;
  }
  std::vector<DecJob> jl;
  for (int i0 = 0; i0 < nfields; i0 += kMaxDecJobs) {
    jl.clear();
    for (int i = i0; i < nfields && i < i0 + kMaxDecJobs; ++i) {
      DecJob j{};
      j.g = P[i].g;
      j.in = P[i].in;
      j.di = P[i].di;
      j.ds = P[i].ds;
      jl.push_back(j);
    }
    int st = launch_huff_jobs(jl.data(), (int)jl.size(), s);
    if (st) return st;
  }
  // reconstructions on a few streams of their own, so that small fields run side by side
  AuxStreams* aux = aux_streams();
  if (int st = aux_fork(aux, s)) return st;
  for (int i = 0; i < nfields; ++i) {
    int st = launch_dec(P[i], mlps[i], nsm, aux->s[i % kAuxStreams], nullptr, kDecRecon);
    if (st) return st;
  }
  if (int st = aux_join(aux, s)) return st;
  std::vector<int> errs((size_t)nfields, 0);
  for (int i = 0; i < nfields; ++i)
    if (cudaMemcpyAsync(&errs[i], P[i].ds.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  prof_collect();
  for (int i = 0; i < nfields; ++i)
    if (errs[i]) return errs[i];
  return PC_OK;
}

int pc_header_info(const void* h_hdr, size_t hdr_bytes, size_t dims_out[3], int* dtype_out, size_t* ws_bytes) {
  Hdr H;
  Geo g;
  int st = parse_header(static_cast<const uint8_t*>(h_hdr), hdr_bytes, H, g);
  if (st) return st;
  if (dims_out)
    for (int i = 0; i < 3; ++i) dims_out[i] = H.dims[i];
  if (dtype_out) *dtype_out = H.dtype;
  if (ws_bytes) *ws_bytes = dec_layout(g, H.m, H.lossless ? 4ull * H.swords : 0ull).total;
  return PC_OK;
}

int pc_decompress(const void* d_in, size_t in_size, void* d_field, size_t field_cap, size_t dims_out[3],
                  int* dtype_out, void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_in || !d_field || !d_ws) return PC_ERR_ARG;
  if (in_size < (size_t)kHdr) return PC_ERR_CORRUPT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the header and the largest FP32 weight section in one read-back
  static thread_local uint8_t hbuf[kHdr + 4 * kMaxW];
  const size_t pre = in_size < sizeof(hbuf) ? in_size : sizeof(hbuf);
  if (cudaMemcpyAsync(hbuf, d_in, pre, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  static thread_local Mlp mlp;
  DecPlan P;
  int st = plan_dec(P, hbuf, pre, d_in, in_size, d_field, field_cap, d_ws, ws_bytes, mlp);
  if (st) return st;
  if (dims_out)
    for (int i = 0; i < 3; ++i) dims_out[i] = P.H.dims[i];
  if (dtype_out) *dtype_out = P.H.dtype;
  const int nsm = sm_count();
  if (nsm <= 0) return PC_ERR_CUDA;
  int r = launch_dec(P, mlp, nsm, s);
  if (r) return r;
  int err = 0;
  if (cudaMemcpyAsync(&err, P.ds.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  prof_collect();
  return err ? err : PC_OK;
}

int pc_compress_host(const void* h_field, const size_t dims[3], int dtype, const pc_params* p, void* h_out,
                     size_t out_cap, size_t* out_size, void* d_field_stage, void* d_out_stage, size_t d_out_cap,
                     void* d_ws, size_t ws_bytes, void* stream) {
  if (!h_field || !h_out || !d_field_stage || !d_out_stage || !dims || !out_size) return PC_ERR_ARG;
  if (dtype != PC_F32 && dtype != PC_F64) return PC_ERR_DTYPE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = dims[0] * dims[1] * dims[2] * (dtype == PC_F64 ? 8 : 4);
  if (cudaMemcpyAsync(d_field_stage, h_field, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return PC_ERR_CUDA;
  size_t sz = 0;
  int st = pc_compress(d_field_stage, dims, dtype, p, d_out_stage, d_out_cap, &sz, d_ws, ws_bytes, stream);
  if (st) return st;
  if (sz > out_cap) return PC_ERR_CAPACITY;
  if (cudaMemcpyAsync(h_out, d_out_stage, sz, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  *out_size = sz;
  return PC_OK;
}

int pc_decompress_host(const void* h_in, size_t in_size, void* h_field, size_t field_cap, size_t dims_out[3],
                       int* dtype_out, void* d_in_stage, size_t d_in_cap, void* d_field_stage, void* d_ws,
                       size_t ws_bytes, void* stream) {
  if (!h_in || !h_field || !d_in_stage || !d_field_stage || !d_ws) return PC_ERR_ARG;
  if (in_size > d_in_cap) return PC_ERR_CAPACITY;
  if (in_size < (size_t)kHdr) return PC_ERR_CORRUPT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the header (and the FP32 weights) straight from the host copy: no read-back
  const size_t pre = in_size < (size_t)(kHdr + 4 * kMaxW) ? in_size : (size_t)(kHdr + 4 * kMaxW);
  static thread_local Mlp mlp;
  DecPlan P;
  int st = plan_dec(P, static_cast<const uint8_t*>(h_in), pre, d_in_stage, in_size, d_field_stage, field_cap, d_ws,
                    ws_bytes, mlp);
  if (st) return st;
  const int nsm = sm_count();
  if (nsm <= 0) return PC_ERR_CUDA;
  if (cudaMemcpyAsync(d_in_stage, h_in, in_size, cudaMemcpyHostToDevice, s) != cudaSuccess) return PC_ERR_CUDA;
  // the field goes to the host in slabs while later slabs are reconstructed
  SlabSink* sink = host_sink(h_field);
  if (!sink) return PC_ERR_CUDA;
  int r = launch_dec(P, mlp, nsm, s, sink);
  if (r) return r;
  const size_t bytes = P.H.dims[0] * P.H.dims[1] * P.H.dims[2] * (P.H.dtype == PC_F64 ? 8 : 4);
  if (!sink->used && cudaMemcpyAsync(h_field, d_field_stage, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PC_ERR_CUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, P.ds.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
  prof_collect();
  if (err) return err;
  if (dims_out)
    for (int i = 0; i < 3; ++i) dims_out[i] = P.H.dims[i];
  if (dtype_out) *dtype_out = P.H.dtype;
  return PC_OK;
}

const char* pc_strerror(int status) {
  switch (status) {
    case PC_OK: return "ok";
    case PC_ERR_ARG: return "bad argument";
    case PC_ERR_DTYPE: return "unsupported dtype";
    case PC_ERR_NONFINITE: return "NaN or Inf in the input";
    case PC_ERR_CAPACITY: return "output or workspace buffer too small";
    case PC_ERR_CORRUPT: return "corrupt compressed stream";
    case PC_ERR_TIMEOUT: return "bounded device wait ran out";
    case PC_ERR_CUDA: return "CUDA runtime error";
    case PC_ERR_EB_RANGE: return "error bound too small for the dtype";
    default: return "unknown status";
  }
}

}  // extern "C"
