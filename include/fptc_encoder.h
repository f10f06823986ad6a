/*
 * fptc_encoder.h -- the FPTC encoder on the GPU, for streams whose samples are
 * already in GPU memory (server-side re-encoding; in the paper the encoder runs
 * on the acquisition device, and fptc_codec.h is its sequential host form).
 * Per stream it computes the windowed DCT-II of Eq. 1 (zero-padded last
 * window, first E bins, FP64), the three-zone quantizer of Sec. 3.2 (Eq. 2,
 * Eq. 3, zone 2 -> level 128) and the SymLen packing of Alg. 1 (Sec. 4.1):
 * canonical Huffman codewords of the domain's code lengths, whole codewords
 * MSB first into 64-bit words, a new word whenever the next codeword does not
 * fit, symlen[w] = codewords in word w.
 *
 * Levels are those of the FP64 coefficient computed as the host encoder does
 * (products and sums rounded separately, in sample order): each bin is computed
 * in compensated FP32 with an error bound and again in FP64 wherever that bound
 * straddles a level boundary.  A CPU that sums in another order may round a
 * coefficient sitting on a boundary to a neighbouring level.  Packing given
 * levels is exact.
 */
#ifndef FPTC_ENCODER_H_
#define FPTC_ENCODER_H_

#include "fptc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fptc_encoder fptc_encoder;

/* Device status flags of an encode (fptc_encoder_status). */
#define FPTC_ENC_FLAG_NO_CODE 1u   /* a level without a codeword in its domain */
#define FPTC_ENC_FLAG_ROOM 2u      /* a stream needed more words than its room */

/* Validates the domains (as fptc_plan_create) and the segments, which use the
 * fptc_segment fields this way:
 *   out_offset  first sample of the stream in d_x (floats),
 *   n_samples   samples S of the stream,
 *   word_offset first word of the room reserved for the stream in d_words and
 *               d_symlen,
 *   n_words     size of that room (words; fptc_word_capacity(domain, S) always
 *               suffices), rooms may not overlap,
 *   domain      index into domains.
 * Uploads the cosine tables (cos(pi/N (n + 1/2) k), host FP64), the canonical
 * codewords and lengths of every domain and the segment table to `device`.
 * Returns FPTC_ERR_INVALID_ARGUMENT (with a message) for bad input,
 * FPTC_ERR_OUT_OF_MEMORY / FPTC_ERR_CUDA on device failures; *enc = NULL then. */
fptc_status fptc_encoder_create(fptc_encoder **enc, int device, const fptc_domain *domains, uint32_t n_domains,
                                const fptc_segment *segments, uint64_t n_segments);

/* Frees the encoder's device memory (synchronizes the device first). NULL is a no-op. */
void fptc_encoder_destroy(fptc_encoder *enc);

/* Sum over segments of W*E (W = ceil(S/N)): the length of a level buffer. */
uint64_t fptc_encoder_levels(const fptc_encoder *enc);

/* Offset of each segment's W*E levels in a level buffer (caller order, packed
 * back to back); offsets holds n_segments values. */
fptc_status fptc_encoder_level_offsets(const fptc_encoder *enc, uint64_t *offsets);

/* Encodes every segment: d_x float32 samples (device), d_words / d_symlen the
 * rooms (device, caller-owned), d_n_words[i] (device, uint64 [n_segments],
 * caller order) receives the words written for segment i.  d_levels: NULL, or
 * a device buffer of fptc_encoder_levels() bytes that receives the levels.
 * Words of a room past d_n_words[i] are left as they were.  Asynchronous on
 * `stream`.  Without d_levels the first such call allocates the encoder's own
 * level buffer (kept until fptc_encoder_destroy); otherwise nothing is
 * allocated.  Problems found on the device (a level with no codeword, a room
 * too small) are reported by fptc_encoder_status; such a stream gets
 * d_n_words[i] = 0 and the contents of its room are undefined. */
fptc_status fptc_encode_device(fptc_encoder *enc, const float *d_x, uint64_t *d_words, uint8_t *d_symlen,
                               uint64_t *d_n_words, uint8_t *d_levels, fptc_stream stream);

/* SymLen packing of given levels (device, fptc_encoder_levels() bytes, the
 * layout of fptc_encoder_level_offsets) into the rooms, as fptc_encode_device
 * does after quantizing. */
fptc_status fptc_pack_device(fptc_encoder *enc, const uint8_t *d_levels, uint64_t *d_words, uint8_t *d_symlen,
                             uint64_t *d_n_words, fptc_stream stream);

/* Synchronizes the device, returns FPTC_ERR_CORRUPT_STREAM if an encode since
 * the last call flagged a segment (flags: FPTC_ENC_FLAG_*, *first_bad: the
 * smallest such segment index), else FPTC_OK; clears the status. */
fptc_status fptc_encoder_status(fptc_encoder *enc, uint32_t *flags, uint64_t *first_bad);

#ifdef __cplusplus
}
#endif

#endif /* FPTC_ENCODER_H_ */
