/*
 * pc.h - C ABI of the GB300 perceptron-predicted, pointwise-relative-error
 * bounded lossy compressor (arXiv 2309.09778).
 *
 * Method (paper sections):
 *   Section III (Eq. 6-12)  relative -> absolute map x -> log2(|x| factor), with a
 *                           positive and a negative factor so that the sign lives
 *                           in the code and needs no extra storage;
 *   Section IV.A-B          prediction of each code from its causal in-block
 *                           neighbours by a three-layer perceptron (leaky ReLU),
 *                           with the Lorenzo predictor as per-block fallback;
 *   Section IV.D            data selection from true (pre-quantized) values, which
 *                           makes prediction parallel; balance points (outliers);
 *   Section IV.A, V (Alg. 1) linear-scaling quantization, Huffman coding and the
 *                           bitstream; decompression inverts every step.
 *
 * Conventions for every entry point:
 *   - Device pointers ("d_") are CUDA global memory of the current device; host
 *     pointers ("h_") are ordinary host memory.  The caller owns every buffer and
 *     the stream.  No entry point allocates device memory: scratch space comes
 *     from the caller's workspace (size from the *_workspace_size calls).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Work is stream-ordered; calls that return a host value (sizes)
 *     synchronize that stream before returning.
 *   - Fields are C-order (row-major) arrays of dims[0] x dims[1] x dims[2]
 *     elements, dims[2] fastest.  1-D and 2-D fields use leading dims of 1.
 *   - Every call returns a status: PC_OK (0) or a negative PC_ERR_* code; no
 *     call aborts the process.  pc_strerror() names a status.
 *   - The library fails loudly: there is no CPU fallback for any step.
 */
#ifndef PC_H
#define PC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PC_OK 0
#define PC_ERR_ARG (-1)        /* bad argument (sizes, shapes, eb outside (0,1), ...) */
#define PC_ERR_DTYPE (-2)      /* dtype not PC_F32 / PC_F64 */
#define PC_ERR_NONFINITE (-3)  /* NaN or Inf in the input field */
#define PC_ERR_CAPACITY (-4)   /* output or workspace buffer too small */
#define PC_ERR_CORRUPT (-5)    /* compressed stream fails validation */
#define PC_ERR_TIMEOUT (-6)    /* a bounded device wait ran out */
#define PC_ERR_CUDA (-7)       /* a CUDA runtime call failed */
#define PC_ERR_EB_RANGE (-8)   /* codes would leave +-2^30 (eb too small for the dtype) */

/* element types */
#define PC_F32 0
#define PC_F64 1

/* predictor forms */
#define PC_PRED_LORENZO 0      /* Lorenzo only (Section IV.A) */
#define PC_PRED_MLP_FP32 1     /* perceptron in FP32 on CUDA cores, Lorenzo per-block fallback */
#define PC_PRED_MLP_BF16 2     /* fixed-point perceptron on the tensor cores (pc_quantize), Lorenzo fallback */

typedef struct {
  double eb_rel;          /* pointwise relative bound b_r, 0 < eb_rel < 1 (Eq. 1) */
  int block[3];           /* compression block shape, product in [2, 4096] (Section IV.C) */
  int pred;               /* PC_PRED_* */
  int stencil;            /* perceptron inputs: 7 (3-D Lorenzo set) or 13 (causal half of 3x3x3) */
  int hidden[2];          /* hidden widths {h1, h2}; h2 = 0 gives the paper's single hidden layer */
  int m;                  /* code bits, 2..16: codes span 0 .. 2^m - 1 (Section IV.C) */
  int s_in;               /* input scale: inputs are codes * 2^-s_in (from pc_train) */
  const float* h_weights; /* host pointer to the perceptron weight blob (pc_mlp_nweights floats):
                             W1[h1][k], b1[h1], W2[h2][h1], b2[h2], W3[hl], b3 (hl = h2 or h1);
                             used by PC_PRED_MLP_FP32 */
  const long long* h_qnet;/* host pointer to the fixed-point network (pc_qnet_len int64, from
                             pc_quantize); used by PC_PRED_MLP_BF16 */
  unsigned long long seed;/* sampling and initialisation seed of the training phase */
  long long train_samples;/* expected number of sampled stencils of the training phase;
                             0 draws 10% of the non-anchor points (Section IV.C) */
  int ndims;              /* 1, 2 or 3 (0: not stated); the leading 3 - ndims dims must be 1 */
  int codebook_n;         /* entries of h_codebook */
  const unsigned int* h_codebook;
                          /* host pointer to a sample codebook (pc_sample_codebook) or NULL.
                             With it, pc_compress runs in one pass over the field: the code
                             words come from this list instead of the field's own histogram,
                             a code the list lacks becomes a balance point, and the container
                             places the bitstream before the balance values (Section IV.C
                             keeps the training phase's Huffman code for compression) */
  int literal;            /* 1: the paper-literal data selection of Section IV.D, an experimental mode
                             (float32 fields, PC_PRED_LORENZO or PC_PRED_MLP_FP32 with weights): every
                             point is predicted from the true values of its neighbours, the decoder
                             predicts from its reconstructions and drifts, so the bound is NOT
                             guaranteed; the container is flagged and decodes with the drift */
  int eq_period;          /* literal mode: every eq_period-th point of a block (raster order) is stored
                             as a deliberate equilibrium point; 0 = none */
  int lossless;           /* 1: the fourth SZ stage of Section IV.A, a lossless LZ77-style pass over the
                             bitstream bytes in independent 16 KiB chunks (not with h_codebook) */
} pc_params;
/*
 * Learned predictor trained inside pc_compress (Section IV.C, V): with
 * pred = PC_PRED_MLP_FP32 and h_weights = NULL, or PC_PRED_MLP_BF16 and
 * h_qnet = NULL, pc_compress first runs the training phase of pc_train on the
 * device (seed, train_samples, the library's 16-model learning-rate x L2 grid)
 * and, for the fixed-point form, pc_quantize; the chosen network (or Lorenzo,
 * when no model beats it) then compresses the field.  The chosen weights come
 * back to the host once, mid-call.  The workspace must then also hold the
 * training buffers (pc_compress_workspace_size accounts for them).
 * Supported shapes: (7, 16, 16) and (13, 32, 32); the FP32 form also
 * (7, 8, 8), (7, 2, 0) and (13, 16, 16).
 */

/* Number of floats in the weight blob for stencil k and hidden widths h1, h2. */
int pc_mlp_nweights(int k, int h1, int h2);

/*
 * Fixed-point form of the perceptron of Section IV.B (the low-precision
 * tensor-core form), bit-reproducible by construction.  Its weights are 8-bit
 * integers, exact in bf16 and f16; the device evaluates it on the tensor cores
 * with 16-bit operands holding 9-bit integer limbs of the inputs and
 * activations and exact FP32 accumulation (tcgen05 with TMEM accumulators in
 * compression, warp-level MMAs along the decoder's wavefronts).
 * The network is an int64 array of pc_qnet_len(k, h1, h2)
 * entries: k, h1, h2, s_in, e1, e2, e3, t1, t2, then W1[h1][k], B1[h1],
 * W2[h2][h1], B2[h2], W3[h2], B3.
 *  - Weights of layer l are integers |W| <= 255 standing for W 2^-e_l.
 *  - Stencil inputs are the centred codes clamped to +-(2^16 - 1).
 *  - Each hidden layer computes A = sum W x + B (exact integer), then
 *    leaky(A) = A >= 0 ? A : A / 16, then H = clamp(rhu(leaky(A) 2^-t), +-(2^15 - 1)),
 *    rhu rounding halves up.
 *  - The output is pred = clamp(rne(A 2^-F), +-2^30), F = e1 + e2 + e3 - t1 - t2;
 *    rne rounds to nearest, ties to even.
 * Supported shapes: (k, h1, h2) = (7, 16, 16) and (13, 32, 32).
 * The network travels in the container's weights section, and decompression
 * checks its ranges (PC_ERR_CORRUPT).
 */
int pc_qnet_len(int k, int h1, int h2);

/*
 * Build the fixed-point network from trained FP32 weights p->h_weights with
 * input scale p->s_in (from pc_train), on the device.
 *  - Weight exponents: e_l is the largest e with max|W_l| 2^e <= 255, kept in
 *    [-30, 30]; W = rint(W_f32 2^e).
 *  - Biases: rint of the f32 bias in the units of its layer's sum, clamped to +-2^40.
 *  - Shifts: each hidden layer's t is the smallest t in [-24, 40] with
 *    max 16 |leaky(A)| 2^-t <= 16 (2^15 - 1). The maximum is over the used
 *    training and validation samples, drawn as by pc_train with the same seed
 *    and thr32.
 * Arguments:
 *   h_qnet_out [out] host, pc_qnet_len(p->stencil, p->hidden[0], p->hidden[1]) int64.
 *   d_ws       workspace of pc_train_workspace_size(dims, dtype, p, thr32, 1) bytes.
 * Errors: PC_ERR_ARG (unsupported shape, missing weights), PC_ERR_CAPACITY, PC_ERR_CUDA.
 */
int pc_quantize(const void* d_field, const size_t dims[3], int dtype, const pc_params* p, unsigned long long seed,
                unsigned int thr32, long long* h_qnet_out, void* d_ws, size_t ws_bytes, void* stream);

/* Upper bound, in bytes, on the compressed size of a field (header, weights,
 * codebook, block table, balance points, bitstream).  0 on bad arguments. */
size_t pc_compress_bound(const size_t dims[3], int dtype, const pc_params* p);

/* Device workspace, in bytes, that pc_compress needs for this field. */
int pc_compress_workspace_size(const size_t dims[3], int dtype, const pc_params* p, size_t* ws_bytes);

/*
 * Compress a device-resident field (Algorithm 1).
 *   d_field   [in]  dims[0]*dims[1]*dims[2] elements of dtype, device memory.
 *   d_out     [out] device buffer of out_cap bytes; receives the container.
 *   out_size  [out] host size_t: container bytes written.
 *   d_ws      [scratch] device workspace of ws_bytes >= pc_compress_workspace_size.
 * The stream is synchronized once, at the end, to read the size and status.
 * A field holds at most 2^32 - 1 points (code counts are 32-bit); larger
 * fields are compressed as independent partitions by the caller.
 * Errors: PC_ERR_ARG (also for more than 2^32 - 1 points), PC_ERR_DTYPE, PC_ERR_NONFINITE, PC_ERR_EB_RANGE,
 * PC_ERR_CAPACITY (out_cap or ws_bytes too small), PC_ERR_CUDA.
 */
int pc_compress(const void* d_field, const size_t dims[3], int dtype, const pc_params* p,
                void* d_out, size_t out_cap, size_t* out_size,
                void* d_ws, size_t ws_bytes, void* stream);

/*
 * Read the fixed 256-byte container header from a host copy (h_hdr, hdr_bytes >= 256):
 * dims, dtype and the decompression workspace size.  Validates magic, version
 * and header CRC; PC_ERR_CORRUPT otherwise.
 */
int pc_header_info(const void* h_hdr, size_t hdr_bytes, size_t dims_out[3], int* dtype_out,
                   size_t* ws_bytes);

/*
 * Decompress a device-resident container (Section V, decompression).
 *   d_in       [in]  in_size bytes of container, device memory.
 *   d_field    [out] device buffer of field_cap bytes; receives the field.
 *   dims_out, dtype_out [out] host.
 *   d_ws       [scratch] device workspace of ws_bytes (see pc_header_info).
 * Reads the header and weights to the host first (one small copy and a
 * stream synchronization), validates everything it reads, and reports a
 * damaged stream as PC_ERR_CORRUPT without faulting.
 */
int pc_decompress(const void* d_in, size_t in_size, void* d_field, size_t field_cap,
                  size_t dims_out[3], int* dtype_out, void* d_ws, size_t ws_bytes, void* stream);

/*
 * Batched compression of nfields fields of uneven shapes and dtypes (the
 * batching of many fields: each field is compressed exactly as pc_compress
 * would, into its own container).  Fields that share dtype, block shape and
 * predictor form (and, for PC_PRED_MLP_FP32, the same h_weights pointer) go
 * through the hot kernel (a4-a9) in one persistent launch over their
 * (field, brick) work list, up to 32 fields per launch; statistics, codebook
 * and packing stay per field.  Every field needs explicit weights (no
 * training inside the batch).  The stream is synchronized once, at the end.
 *   dims      [in]  host, 3 * nfields sizes (field i: dims[3i .. 3i+2]).
 *   dtypes, params [in] host, nfields each.
 *   d_out     [out] container i starts at d_out + offsets[i] (offsets are
 *                   the 256-byte aligned prefix sums of pc_compress_bound).
 *   offsets   [out] host, nfields + 1;  sizes [out] host, container bytes.
 *   d_ws      [scratch] pc_compress_batch_workspace_size bytes.
 * Errors: as pc_compress (the first failing field's status); PC_ERR_ARG when a
 * field asks for training.
 */
int pc_compress_batch_workspace_size(int nfields, const size_t* dims, const int* dtypes, const pc_params* params,
                                     size_t* ws_bytes, size_t* out_bytes);
int pc_compress_batch(int nfields, const void* const* d_fields, const size_t* dims, const int* dtypes,
                      const pc_params* params, void* d_out, size_t out_cap, size_t* offsets, size_t* sizes,
                      void* d_ws, size_t ws_bytes, void* stream);

/*
 * Batched decompression of nfields containers held in one device buffer
 * (container i at d_in + offsets[i], sizes[i] bytes) into d_fields[i]
 * (field_caps[i] bytes each).  Reads every header back in one
 * synchronization, prepares every field's decoder tables, runs the Huffman
 * decoders of up to 32 fields in one launch, then the reconstructions on four
 * streams of the library's own (created on first use, one set per host thread
 * and device, and kept) that the caller's stream waits for; synchronizes once
 * more at the end.  The workspace size comes
 * from the 256-byte headers (host copies) through
 * pc_decompress_batch_workspace_size.
 */
int pc_decompress_batch_workspace_size(int nfields, const void* const* h_headers, size_t* ws_bytes);
int pc_decompress_batch(int nfields, const void* d_in, const size_t* offsets, const size_t* sizes,
                        void* const* d_fields, const size_t* field_caps, void* d_ws, size_t ws_bytes, void* stream);

/*
 * Decompression that allocates nothing, for callers that cannot obtain device
 * memory at the point of the call: hosts whose device-memory budget is fixed
 * up front, or plugins given only an input and an output buffer by a
 * framework that owns every allocation.
 * The paper has no counterpart: this is a deployment convenience.
 * Same arguments and results as pc_decompress, without the workspace: the
 * scratch space is a fixed 32 MiB array compiled into the library, held on
 * every GPU that loads it until the process exits (enough for fields up to
 * about 16 million points with 8x8x8 blocks).  Returns PC_ERR_CAPACITY,
 * before launching anything, when the container needs more scratch than
 * that.  Like pc_decompress, the call reads the header back to the host and
 * synchronizes the stream.  The first call on each device looks up the
 * array's device address.  All calls share the array: calls that overlap on
 * the GPU race and must be serialized by the caller.
 */
int pc_decompress_noalloc(const void* d_in, size_t in_size, void* d_field, size_t field_cap,
                          size_t dims_out[3], int* dtype_out, void* stream);

/*
 * End-to-end forms with HOST buffers: copy the input host -> device, run the
 * device call, copy the result device -> host, synchronize.  The caller passes
 * device staging buffers (no device memory is allocated): d_field_stage holds
 * the field (field bytes), d_out_stage the container (d_out_cap bytes).
 * h_field and h_out should be pinned for full copy speed.
 * pc_decompress_host reads the header from the host copy (no read-back) and,
 * for fields of at least 16 block planes, copies the field out in 8 slabs of
 * whole block planes on a stream of its own while later slabs are being
 * reconstructed; that stream and its events are created on first use, one set
 * per host thread and device, and kept.
 */
int pc_compress_host(const void* h_field, const size_t dims[3], int dtype, const pc_params* p,
                     void* h_out, size_t out_cap, size_t* out_size,
                     void* d_field_stage, void* d_out_stage, size_t d_out_cap,
                     void* d_ws, size_t ws_bytes, void* stream);
int pc_decompress_host(const void* h_in, size_t in_size, void* h_field, size_t field_cap,
                       size_t dims_out[3], int* dtype_out,
                       void* d_in_stage, size_t d_in_cap, void* d_field_stage,
                       void* d_ws, size_t ws_bytes, void* stream);

/*
 * Training phase (Section IV.C) on the device: sample stencils (rate thr32 / 2^32
 * of non-anchor points, 10% by default), split 8:2, train nmodels copies of the
 * Lorenzo-initialised perceptron for one epoch of minibatch SGD (batch 256) with
 * learning rates lrs[i] and L2 weights lams[i], score each and Lorenzo on the
 * validation samples by residual bit length, and choose.
 *   h_weights_out [out] host, nmodels * pc_mlp_nweights floats (every trained model).
 *   s_in_out      [out] input scale exponent.
 *   chosen_out    [out] index of the chosen model, -1 if Lorenzo scored best.
 *   h_costs       [out] host, nmodels + 1 validation costs (last = Lorenzo), may be NULL.
 * Uses p->block, p->stencil, p->hidden, p->m and p->eb_rel.
 */
int pc_train_workspace_size(const size_t dims[3], int dtype, const pc_params* p, unsigned int thr32,
                            int nmodels, size_t* ws_bytes);
int pc_train(const void* d_field, const size_t dims[3], int dtype, const pc_params* p,
             unsigned long long seed, unsigned int thr32, int nmodels,
             const float* h_lrs, const float* h_lams,
             float* h_weights_out, int* s_in_out, int* chosen_out, unsigned long long* h_costs,
             void* d_ws, size_t ws_bytes, void* stream);

/*
 * The training phase with the paper's model selection (Section IV.C): the
 * models are trained as by pc_train, then every model and Lorenzo is scored
 * by simulating compression on the validation samples -- residuals quantized
 * with p->m code bits (code k + R, or a balance point), Huffman-coded with the
 * code of their own histogram (as the compressor builds it), plus the stored
 * value (32 or 64 bits) of every balance point -- and the smallest simulated
 * size wins (Lorenzo unless strictly beaten).  Then m is chosen by the
 * coverage rule: coverage(m) is the share of validation residuals with
 * |k| <= 2^(m-1) - 1, and m in 2..16 is taken with coverage closest to 50%
 * when eb_rel < 1.5%, to 80% otherwise (the larger m on a tie).
 *   h_sizes [out] host, nmodels + 1 simulated sizes in bits (last = Lorenzo), may be NULL.
 *   m_out   [out] the chosen code bits.
 * Workspace: pc_train_workspace_size.  Other arguments and errors as pc_train.
 */
int pc_train_select(const void* d_field, const size_t dims[3], int dtype, const pc_params* p,
                    unsigned long long seed, unsigned int thr32, int nmodels, const float* h_lrs,
                    const float* h_lams, float* h_weights_out, int* s_in_out, int* chosen_out,
                    unsigned long long* h_sizes, int* m_out, void* d_ws, size_t ws_bytes, void* stream);

/*
 * Sample codebook (Section IV.C): the training phase draws its validation
 * samples (seed, thr32, as pc_train), quantizes their residuals under the
 * predictor of p -- the FP32 weights p->h_weights (stencil, hidden, s_in), or
 * Lorenzo when p->pred is PC_PRED_LORENZO -- at p->m code bits, and builds the
 * Huffman code of their histogram.  The paper averages the frequencies per
 * block; dividing every count by the block count leaves the Huffman code
 * unchanged, so the totals are used.  Symbol 0 (the balance-point marker)
 * counts at least once so that balance points stay codable.  A code the
 * sample never saw has no code word and compresses as a balance point;
 * span_fill = 1 gives every code between the smallest and the largest sampled
 * code a code word (counted once), so that only codes beyond the sampled span
 * do (not in the paper: a small validation sample of a wide residual
 * distribution misses many codes inside its span).
 *   h_codebook_out [out] host, up to 2^m entries: sym | length << 16, in the
 *                  order the container stores them (most frequent first).
 *   n_out          [out] number of entries.
 * Pass the list as pc_params.h_codebook / codebook_n to compress in one pass.
 * Workspace: pc_train_workspace_size(dims, dtype, p, thr32, 1).
 * Errors: PC_ERR_ARG (unsupported shape, missing weights), PC_ERR_CAPACITY, PC_ERR_CUDA.
 */
int pc_sample_codebook(const void* d_field, const size_t dims[3], int dtype, const pc_params* p,
                       unsigned long long seed, unsigned int thr32, int span_fill, unsigned int* h_codebook_out,
                       int* n_out, void* d_ws, size_t ws_bytes, void* stream);

/* Diagnostics for tests: offsets (bytes) of the per-point codes (u16, block-strided,
 * nblocks * block volume), per-block perceptron flags (u8) and the code histogram
 * (u64, 2^m) inside a compression workspace after pc_compress returns. */
int pc_compress_workspace_layout(const size_t dims[3], int dtype, const pc_params* p,
                                 size_t* off_codes, size_t* off_nnflag, size_t* off_hist);

/*
 * Per-kernel timing (tracing).  pc_profile_enable(1) makes every following
 * pc_compress / pc_decompress record a CUDA event pair around each of its
 * kernel launches on the call's stream; the durations are added up per stage
 * once the call has synchronized.  pc_profile_read copies up to n stage sums
 * (milliseconds of device time) and launch counts, then clears them; it
 * returns the number of stages.  pc_profile_stage_name names stage i.
 * Events are created once per process on first enable (no device memory).
 */
int pc_profile_enable(int on);
int pc_profile_read(double* ms, long long* launches, int n);
const char* pc_profile_stage_name(int i);

/* Human-readable name of a status code. */
const char* pc_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* PC_H */
