/*
 * CPU oracle for the perceptron-predicted, pointwise-relative-error-bounded
 * compressor (arXiv 2309.09778).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path; both sides follow the same written specification.
 *
 * Everything here is plain, slow, single-threaded C.  Floating-point work is
 * IEEE round-to-nearest with FMA contraction disabled at compile time; where a
 * fused multiply-add is part of the specification it is written as fmaf/fma.
 */
#ifndef PC_ORACLE_H
#define PC_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_DTYPE (-2)
#define ORC_ERR_NONFINITE (-3)
#define ORC_ERR_CAPACITY (-4)
#define ORC_ERR_CORRUPT (-5)
#define ORC_ERR_EB_RANGE (-8)

#define ORC_F32 0
#define ORC_F64 1

#define ORC_PRED_LORENZO 0
#define ORC_PRED_MLP 1
#define ORC_PRED_MLP_BF16 2  /* fixed-point perceptron on bf16 tensor-core operands */
#define ORC_PRED_MLP64 3     /* the FP32 weights evaluated in FP64 (reporting only) */

typedef struct {
  int dtype;
  double eb, abs_min, abs_max;
  int trivial;           /* field has no normal value */
  double step64;         /* 2 b_a in double */
  float step32, inv32, ebdn32;
  double stepd, invd, ebdnd;
  int32_t Kp, Kn, Zq, S;
} orc_consts;

typedef struct {
  double eb;
  int block[3];
  int pred;              /* ORC_PRED_* */
  int stencil;           /* 7 or 13 */
  int h1, h2;            /* hidden widths; h2 == 0: one hidden layer */
  int m;                 /* code bits; radius R = 2^(m-1) */
  int s_in;              /* input scale: u = v * 2^-s_in */
  const float* weights;  /* MLP weight blob, NULL for Lorenzo only */
  const int64_t* qnet;   /* fixed-point network (ORC_PRED_MLP_BF16), see orc_qnet_len */
  const uint32_t* codebook; /* sample codebook (sym | len << 16, container order) or NULL: see
                               orc_compress; NULL builds the code of the field's own histogram */
  int codebook_n;        /* entries of codebook */
  int literal;           /* 1: the paper-literal data selection (Section IV.D), float32 only, FP32
                            perceptron or Lorenzo: see orc_compress */
  int eq_period;         /* literal mode: every eq_period-th point of a block (raster order) is a
                            deliberate equilibrium point; 0 = none */
  int lossless;          /* 1: the lossless back-end stage over the bitstream bytes (orc_lz_encode) */
} orc_params;

/* container flag (header offset 228): the bitstream section precedes the
 * balance-point values (the layout of a compression with a sample codebook) */
#define ORC_FLAG_STREAM_FIRST 1u
/* container flag: codes of the paper-literal data selection (decoded serially, with drift);
 * header offset 232 holds the equilibrium-point period */
#define ORC_FLAG_LITERAL 4u
/* container flag: the bitstream section holds the lossless stage's chunks
 * (header offset 240: the section's bytes) */
#define ORC_FLAG_LOSSLESS 8u
#define ORC_LZ_CHUNK 16384

typedef struct {
  int32_t* dq;           /* [N] integer log codes, field order */
  uint8_t* ok;           /* [N] per-point bound check */
  uint16_t* codes;       /* [nblocks * bvol] block-strided codes, slot 0 (anchor) = 0 */
  uint8_t* nnflag;       /* [nblocks] 1 = block used the perceptron */
  uint64_t* hist;        /* [2^m] code histogram */
  uint8_t* lens;         /* [2^m] Huffman code lengths */
} orc_dump;

#endif
