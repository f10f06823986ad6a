/*
 * fptc.h -- C ABI of the FPTC server-side batch decoder for one GB300 GPU (sm_103a).
 *
 * FPTC ("FPTC: A Fast Parallel Transform-based Codec for Efficient Asymmetric
 * Signal Compression", arXiv 2605.01086) compresses a signal by a windowed
 * DCT-II (Sec. 3.1, Eq. 1), a hybrid three-zone 8-bit quantizer (Sec. 3.2,
 * Eq. 2, Eq. 3) and length-limited canonical Huffman codes packed into 64-bit
 * words with a per-word symbol count, the SymLen format (Sec. 3.3, Sec. 4.1,
 * Alg. 1).  This library is the decompression side (Sec. 4.2): compressed
 * streams already in GPU memory are Huffman-decoded, dequantized, inverse
 * transformed and written as float32 samples to GPU memory (the timed region of
 * Sec. 5.1).
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are device pointers on the plan's device; h_* are host
 *    pointers.  The caller owns every buffer it passes; the library never frees
 *    or keeps them past the call.
 *  - fptc_stream is the CUDA stream type (interchangeable with cudaStream_t and
 *    CUstream); NULL means the legacy default stream.
 *  - Decode calls are asynchronous on the stream, never allocate and never
 *    synchronize, so they can be captured in a CUDA graph.  One plan serves one
 *    stream at a time (its index scratch is per plan).
 *  - Errors visible from arguments and metadata are returned at once.  Errors
 *    in the compressed payload are found on the device: they set a sticky
 *    status in the plan (read by fptc_plan_device_status), writes stay inside
 *    the offending segment's output range, and no kernel traps.
 *
 * Bitstream format (the readings this library shares with its encoder):
 *  - words: uint64, codewords MSB-first, shift = 64 - bit_size - code_len
 *    (Alg. 1); unused low bits are padding; symlen[w] (uint8, <= 64) = number
 *    of codewords in word w; a codeword never straddles two words (Sec. 4.1).
 *  - codes: canonical in (length, symbol) order starting from 0 (the DEFLATE
 *    rule), built from the 256 code lengths of the domain (Sec. 3.3).
 *  - symbols: one 8-bit level per retained coefficient, window-major
 *    (E levels of window 0, then window 1, ...); W = ceil(S / N) windows, the
 *    last one zero-padded by the encoder.
 *  - levels: zone 0 (bins [0, B1)): 128 = 0; L > 128 -> +(A0/mu)((1+mu)^((L-128)/127) - 1);
 *    L < 128 -> -(A0/mu)((1+mu)^((128-L)/128) - 1)  (inverse of Eq. 2).
 *    zone 1 (bins [B1, B2)): 128 = 0; L >= 129 -> d1 + (L-129)/126 (A1-d1);
 *    L <= 127 -> -(d1 + (127-L)/127 (A1-d1)), d1 = alpha1 A1 (inverse of Eq. 3).
 *    zone 2 (bins [B2, E)) and bins [E, N): 0 (Sec. 3.2.3, Sec. 3.1).
 *    A zone whose scale is <= 1e-30 reconstructs 0.
 *  - samples: x[n] = C[0]/2 + sum_{k=1}^{E-1} C[k] cos(pi/N (n+1/2) k), the
 *    inverse of Eq. 1; window w gives samples [wN, wN+N) of its segment, cut at S.
 */
#ifndef FPTC_H_
#define FPTC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPTC_ABI_VERSION 1u

typedef enum fptc_status {
  FPTC_OK = 0,
  FPTC_ERR_INVALID_ARGUMENT = 1, /* bad parameter, metadata or pointer */
  FPTC_ERR_UNSUPPORTED = 2,      /* valid, but not handled by the chosen path */
  FPTC_ERR_OUT_OF_MEMORY = 3,    /* device or host allocation failed (plan creation only) */
  FPTC_ERR_CUDA = 4,             /* a CUDA runtime call failed; see fptc_last_error_message */
  FPTC_ERR_CORRUPT_STREAM = 5    /* the device found a malformed payload (sticky plan status) */
} fptc_status;

struct CUstream_st;
typedef struct CUstream_st *fptc_stream;

/* One signal domain: the parameters of Table 1 plus the prebuilt structures the
 * encoder and decoder share (Sec. 3, Fig. 4): the per-zone scales A_z and the
 * canonical Huffman code lengths. */
typedef struct fptc_domain {
  uint32_t N;              /* window size (DCT_SIZE), 4..128 */
  uint32_t E;              /* retained coefficients (ENCODED_COEFFS), 1..N */
  uint32_t B1, B2;         /* zone boundaries, 0 <= B1 <= B2 <= E */
  double mu;               /* mu-law strength (MU_COMPANDING), > 0 */
  double alpha1;           /* zone-1 deadzone ratio (DEAD_RATIO_ZONE1), 0..1 */
  double scale[3];         /* A_0, A_1 (A_2 unused: zone 2 is all zero) */
  uint32_t lmax;           /* maximum code length L_max, 1..16 */
  uint8_t code_len[256];   /* code length per level; 0 = level has no code */
} fptc_domain;

/* One compressed stream of the batch (host metadata). */
typedef struct fptc_segment {
  uint64_t word_offset;  /* first word of the stream in the batch word/symlen buffers */
  uint64_t n_words;      /* number of words (and symlen bytes) of the stream */
  uint64_t n_samples;    /* S, samples to reconstruct */
  uint64_t out_offset;   /* first output float of the stream in d_out */
  uint32_t domain;       /* index into the plan's domains */
  uint32_t reserved;     /* must be 0 */
} fptc_segment;

typedef enum fptc_idct {
  FPTC_IDCT_FP32 = 0,    /* FP32 FMAs on the CUDA cores */
  FPTC_IDCT_TF32 = 1,    /* tensor cores (tcgen05, kind::tf32), operands rounded to TF32, FP32 accumulate */
  FPTC_IDCT_BF16X3 = 2,  /* tensor cores, hi/lo BF16 split, three products (hi*hi + lo*hi + hi*lo) */
  FPTC_IDCT_TF32X3 = 3   /* tensor cores, big/small TF32 split, three products */
} fptc_idct;

typedef enum fptc_schedule {
  FPTC_SCHEDULE_PERSISTENT = 0,  /* one persistent launch over every tile of the batch */
  FPTC_SCHEDULE_PER_SEGMENT = 1, /* plain: one set of launches per segment */
  FPTC_SCHEDULE_THREE_KERNEL = 2 /* the GPU design of Sec. 4.2, for comparison: per-word offsets in a
                                    global array, one thread per word writing the levels to a global
                                    byte array, one thread per output sample for dequantization and
                                    inverse DCT.  The plan owns a 4-byte-per-word offset array and a
                                    level array (unless levels are passed); FP32 transform only */
} fptc_schedule;

typedef enum fptc_kernel {
  FPTC_KERNEL_AUTO = 0,        /* warp-tile if every domain has N in [4, 128] (and their tables fit),
                                  else generic */
  FPTC_KERNEL_GENERIC = 1,     /* any N, E: one block per tile, basis through L1 */
  FPTC_KERNEL_BLOCK_TILE = 2,  /* N = 32, E = 16: one block per tile, pipelined */
  FPTC_KERNEL_WARP_TILE = 3,   /* one warp per tile, no block barriers: N = 32, E = 16 (128-window tiles),
                                  or any N in [4, 128] in every domain (several N in one batch; N not a
                                  power of two stores with the lanes instead of TMA), any E <= N (tiles
                                  of about 2048 symbols); at most 8 domains */
  FPTC_KERNEL_TENSOR = 4       /* tensor-core transform, chosen by idct != FPTC_IDCT_FP32: N = 32, E = 16
                                  in every domain, or one (N, E) in {(32, 32), (64, 32), (128, 32),
                                  (128, 64)} shared by every domain */
} fptc_kernel;

typedef struct fptc_plan_options {
  uint32_t idct;          /* fptc_idct */
  uint32_t schedule;      /* fptc_schedule */
  uint32_t tile_samples;  /* target output samples per tile (whole windows) of the block-tile and generic
                             kernels; 0 = 8192 for the block-tile kernel, else 4096.  The warp-tile and
                             tensor-core kernels fix their tiles: 128 windows at N = 32, E = 16; at other
                             shapes about 2048 symbols in whole 1024-sample steps (at most 8) */
  uint32_t threads;       /* threads per CTA: 128, 256 or 512 (also 768, 896, 1024 for the warp-tile kernel
                             at N = 32, E = 16; 256, 512 or 768 for it at other shapes; 384, 640, 768 or
                             896 for the tensor-core kernel at N = 32, E = 16, whose other shapes fix their
                             own); 0 = 256, or for the warp-tile kernel 896 where its shared memory fits
                             (28 warps, no register spills), else the most that fit (at most 512 at other
                             shapes), and for the tensor-core kernel the most that fit shared and tensor
                             memory (896; 640 for its 3xTF32 form); a count that does not fit is refused
                             with FPTC_ERR_UNSUPPORTED */
  uint32_t ctas_per_sm;   /* persistent CTAs per SM; 0 = as many as fit */
  uint32_t kernel;        /* fptc_kernel: which decode kernel; 0 = choose */
  uint32_t reserved[2];   /* must be 0 */
} fptc_plan_options;

typedef struct fptc_plan fptc_plan;

typedef struct fptc_plan_info {
  uint64_t n_segments;
  uint64_t n_tiles;
  uint64_t n_chunks;            /* index work units (chunks of at most 496 words) */
  uint64_t words_extent;        /* max(word_offset + n_words): minimum word/symlen buffer length */
  uint64_t out_extent;          /* max(out_offset + n_samples): minimum output length in floats */
  uint64_t n_samples_total;
  uint64_t n_words_total;
  uint64_t n_levels_total;      /* sum of W*E: length of d_levels / d_grad_coeffs */
  uint64_t device_bytes;        /* device memory owned by the plan */
  uint32_t n_domains;
  uint32_t device;
  uint32_t sm_count;
  uint32_t threads;
  uint32_t grid;                /* persistent CTAs */
  uint32_t ctas_per_sm;
  uint32_t idct;
  uint32_t schedule;
  uint32_t kernel;              /* fptc_kernel in use (never AUTO) */
  uint32_t smem_bytes;          /* dynamic shared memory per CTA of the decode kernel */
} fptc_plan_info;

/* Validates the domains (Table 1 ranges, Kraft inequality of the code lengths)
 * and the segments (domain index, word count consistent with W*E symbols of at
 * most 64 per word, non-overlapping outputs), builds the per-domain decode
 * lookup tables (2^lmax entries, Sec. 3.3) and reconstruction tables (computed
 * in FP64, stored as FP32), lays out the tile queue, and uploads all of it to
 * `device`.  On success *plan owns that device memory until fptc_plan_destroy.
 * Returns FPTC_ERR_INVALID_ARGUMENT, FPTC_ERR_UNSUPPORTED, FPTC_ERR_OUT_OF_MEMORY
 * or FPTC_ERR_CUDA on failure, with *plan set to NULL. opts may be NULL. */
fptc_status fptc_plan_create(fptc_plan **plan, int device, const fptc_domain *domains, uint32_t n_domains,
                             const fptc_segment *segments, uint64_t n_segments, const fptc_plan_options *opts);

/* Frees the plan's device memory (synchronizes the device first). NULL is a no-op. */
void fptc_plan_destroy(fptc_plan *plan);

fptc_status fptc_plan_get_info(const fptc_plan *plan, fptc_plan_info *info);

/* Offsets (in bytes of d_levels / elements of d_grad_coeffs) of each segment's
 * W*E block, in the caller's segment order; offsets must hold n_segments values. */
fptc_status fptc_plan_level_offsets(const fptc_plan *plan, uint64_t *offsets);

/* Decodes every segment of the plan (Sec. 4.2: SymLen index, Huffman decode,
 * dequantization, inverse transform, window reassembly) and writes float32
 * samples to d_out[out_offset .. out_offset + S) of each segment.
 *   d_words   uint64 [words_extent], 8-byte aligned
 *   d_symlen  uint8  [words_extent]
 *   d_out     float  [out_extent], 16-byte aligned; other floats are not touched
 *   d_levels  NULL, or uint8 [n_levels_total]: also store the decoded levels
 *   d_scale   NULL (use the plan's A_z), or float [n_domains * 3]: A_0, A_1, A_2 per
 *             domain, read on the device at run time (differentiable decoding)
 * Asynchronous on `stream`; allocates nothing. */
fptc_status fptc_decode_batch(fptc_plan *plan, const uint64_t *d_words, const uint8_t *d_symlen, float *d_out,
                              uint8_t *d_levels, const float *d_scale, fptc_stream stream);

/* The stages of fptc_decode_batch run separately, for per-stage timing:
 * FPTC_STAGE_INDEX runs the SymLen index kernels (symlen scan into chunk
 * offsets, symbol-count check, and for the block-tile and generic kernels the
 * start of every tile), FPTC_STAGE_DECODE the fused decode kernel, which reads
 * what the last index stage of this plan wrote (so d_symlen must be unchanged
 * since).
 * stages = FPTC_STAGE_INDEX | FPTC_STAGE_DECODE is fptc_decode_batch. */
#define FPTC_STAGE_INDEX 1u
#define FPTC_STAGE_DECODE 2u
/* Plans of schedule FPTC_SCHEDULE_THREE_KERNEL only (the paper's lossless and
 * lossy kernels, Sec. 4.2, whose run-time split Sec. 6 reports): the decode
 * stage's two halves on their own.  FPTC_STAGE_LOSSLESS decodes every word's
 * codewords into the plan's global level array; FPTC_STAGE_LOSSY dequantizes and
 * inverse transforms that array into d_out (it reads what the last lossless
 * stage of this plan wrote).  FPTC_STAGE_DECODE = both.  Other schedules fuse
 * the two halves in one kernel and return FPTC_ERR_UNSUPPORTED for these bits. */
#define FPTC_STAGE_LOSSLESS 4u
#define FPTC_STAGE_LOSSY 8u
fptc_status fptc_decode_stages(fptc_plan *plan, const uint64_t *d_words, const uint8_t *d_symlen, float *d_out,
                               uint8_t *d_levels, const float *d_scale, uint32_t stages, fptc_stream stream);

/* Adjoint of dequantize + inverse transform + window reassembly for a loss L
 * with dL/dx = d_grad_out (same layout as d_out).  For each window and bin k < E:
 *   g_C[k] = sum_n g_x[n] * (1/2 if k = 0 else cos(pi/N (n+1/2) k)), samples past S contribute 0,
 * written to d_grad_coeffs (NULL to skip; float [n_levels_total], level layout), and
 *   d_grad_scale[d*3 + z] = sum over bins of zone z of domain d of g_C * dC/dA_z
 * (double, overwritten; the reconstruction is linear in A_z so dC/dA_z is the
 * reconstruction at A_z = 1; entry z = 2 is 0).  The per-term products are FP32,
 * the reduction FP64.  d_levels: the levels saved by fptc_decode_batch, or NULL
 * to decode them again from d_words / d_symlen.  d_scale as in fptc_decode_batch.
 * Asynchronous on `stream`; allocates nothing. */
fptc_status fptc_decode_backward(fptc_plan *plan, const uint64_t *d_words, const uint8_t *d_symlen,
                                 const uint8_t *d_levels, const float *d_scale, const float *d_grad_out,
                                 float *d_grad_coeffs, double *d_grad_scale, fptc_stream stream);

/* End-to-end decode from host memory: copies h_words / h_symlen (words_extent
 * entries each) into the caller's device buffers, decodes, and copies the
 * samples of every segment back into h_out (out_extent floats).  The work is
 * split in up to 16 pieces of about equal output in output order: a piece's
 * words are uploaded on an internal stream, indexed and decoded on `stream`,
 * and copied back on one of four internal streams, so uploads, decoding and
 * copies back of different pieces overlap (when the words are not laid out in
 * output order, every word is uploaded before the first piece decodes).  Host
 * buffers should be page-locked for full speed.  Returns after h_out holds the
 * result (it synchronizes). */
fptc_status fptc_decode_host(fptc_plan *plan, const uint64_t *h_words, const uint8_t *h_symlen, float *h_out,
                             uint64_t *d_words, uint8_t *d_symlen, float *d_out, fptc_stream stream);

/* Synchronizes the device, then returns FPTC_ERR_CORRUPT_STREAM if any decode
 * since the last call found a malformed payload (and clears the status), else
 * FPTC_OK.  *flags (optional) receives the OR of FPTC_FLAG_* values and
 * *first_bad_segment (optional) the smallest caller index of a bad segment, or
 * UINT64_MAX. */
#define FPTC_FLAG_SYMLEN_RANGE 1u   /* symlen[w] > 64 */
#define FPTC_FLAG_BIT_OVERRUN 2u    /* codewords ran past bit 64 of a word */
#define FPTC_FLAG_INVALID_CODE 4u   /* a bit pattern that is no codeword (incomplete code) */
#define FPTC_FLAG_SYMBOL_COUNT 8u   /* sum of symlen over a segment != W*E */
#define FPTC_FLAG_TIMEOUT 16u       /* a bounded wait on a tensor-core completion barrier gave up */
fptc_status fptc_plan_device_status(fptc_plan *plan, uint32_t *flags, uint64_t *first_bad_segment);

/* Times the candidate tile sizes, CTA sizes and occupancies on the caller's
 * buffers (each candidate decoded `trials` times after one warm-up, CUDA events
 * on `stream`) and keeps the fastest in the plan; *best (optional) receives it
 * and *best_ms its median time.  Synchronizes.  Output buffers are overwritten
 * with valid decodes. */
fptc_status fptc_plan_autotune(fptc_plan *plan, const uint64_t *d_words, const uint8_t *d_symlen, float *d_out,
                               uint32_t trials, fptc_stream stream, fptc_plan_options *best, float *best_ms);

/* Allocation-free decode of ONE stream, for callers that cannot allocate device
 * memory when they decode (inside a framework's memory pool or an allocator
 * callback, where a cudaMalloc would re-enter the allocator; serving paths that
 * forbid allocation after start-up; processes whose device memory another
 * runtime has reserved).  The paper has no counterpart: it is an interface
 * convenience, not part of the method.
 * Same result as a plan with one segment (word_offset 0, out_offset 0) and the
 * generic kernel: index kernels + decode kernel of Sec. 4.2, samples written to
 * d_out[0 .. n_samples).  All working memory (domain tables, records, index
 * scratch, status word) is one file-scope device array of about 2 MB that
 * every device which loads the library keeps until exit; nothing is allocated
 * and no library routine that allocates is called.  The small tables reach
 * the array as the argument of a set-up kernel launched on `stream` (no
 * host-to-device copy; no host memory is read after the call returns).
 * Limits: n_samples <= 67,108,864 and domain->lmax <= 12, else
 * FPTC_ERR_UNSUPPORTED with a message.  Device-side stream errors are not
 * reported by this call (decode with a plan for that).
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress).  The first call on a device also loads this
 * library's device code there (lazy module loading), and that load can
 * allocate device memory: make one call on each device at start-up, before
 * the phase that must not allocate and before any stream capture.  Every call
 * shares the array, so calls whose work overlaps on the GPU (different
 * streams, or other host threads) race; serialize them.  Asynchronous on
 * `stream`. */
fptc_status fptc_decode_stream_noalloc(const fptc_domain *domain, const uint64_t *d_words, const uint8_t *d_symlen,
                                       uint64_t n_words, uint64_t n_samples, float *d_out, fptc_stream stream);

/* Runs, on its own, the bounded wait that every tensor-core and TMA
 * completion wait of the decode kernels uses: one CTA on `device` waits on an
 * mbarrier in its shared memory, sleeping between tests; the wait gives up
 * after 1 s of GPU global time, and the kernel then sets FPTC_FLAG_TIMEOUT in
 * a status word, as the decode kernels do in their plan status.  arrive != 0:
 * one thread arrives on the barrier first (the wait completes, *flags = 0);
 * arrive == 0: nothing arrives (*flags = FPTC_FLAG_TIMEOUT after about 1 s).
 * Either way the kernel returns and the context stays usable.  Synchronous;
 * allocates and frees 4 bytes of device memory.  Errors: NULL flags
 * (FPTC_ERR_INVALID_ARGUMENT), CUDA errors (FPTC_ERR_CUDA). */
fptc_status fptc_check_bounded_wait(int device, int arrive, uint32_t *flags);

/* Kernel launches of one fptc_decode_batch call with the plan's current settings. */
uint32_t fptc_plan_launches_per_decode(const fptc_plan *plan);

/* sizeof of the ABI structs, for bindings that mirror them:
 * 0 = fptc_domain, 1 = fptc_segment, 2 = fptc_plan_options, 3 = fptc_plan_info; other = 0. */
uint64_t fptc_struct_size(uint32_t which);

const char *fptc_status_string(fptc_status status);
/* Text of the last error of this thread (empty if none). */
const char *fptc_last_error_message(void);
uint32_t fptc_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FPTC_H_ */
