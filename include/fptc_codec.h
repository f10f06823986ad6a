/*
 * fptc_codec.h -- host side of the FPTC codec: the prebuilt per-domain
 * structures (Sec. 3.3, Fig. 4) and the sequential single-pass encoder
 * (Sec. 4.1, Alg. 1).  In the paper the encoder runs on the acquisition device;
 * here it produces the compressed streams the GPU decoder consumes.  These
 * calls run on the CPU and touch no GPU.
 */
#ifndef FPTC_CODEC_H_
#define FPTC_CODEC_H_

#include "fptc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Checks one domain: 4 <= N <= 128, 1 <= E <= N, B1 <= B2 <= E, mu > 0,
 * 0 <= alpha1 <= 1, 1 <= lmax <= 16, every code length <= lmax, Kraft sum
 * <= 1 and at least one level with a code.  Returns FPTC_OK or
 * FPTC_ERR_INVALID_ARGUMENT (detail in fptc_last_error_message). */
fptc_status fptc_validate_domain(const fptc_domain *domain);

/* Builds the decode table of Sec. 3.3: 2^lmax uint16 entries, entry p = level |
 * (code length << 8) of the codeword that is a prefix of the lmax-bit pattern p,
 * or 0 where no codeword matches (only possible for an incomplete code).
 * table must hold 1 << lmax entries. */
fptc_status fptc_build_decode_table(const fptc_domain *domain, uint16_t *table);

/* Canonical codewords (Sec. 3.3; DEFLATE order) of the domain's code lengths. */
fptc_status fptc_canonical_codes(const fptc_domain *domain, uint32_t *codes /* 256 */);

/* Trains the prebuilt structures of one domain from representative signals
 * (Sec. 3.2.1, Sec. 3.3): A_0 and A_1 = the `percentile` (nearest rank) of |c|
 * over every training window and every bin of the zone; then the histogram of
 * the quantized training coefficients (+1 on each of the 256 counts) and
 * length-limited optimal code lengths by package-merge.  On input the domain's
 * N, E, B1, B2, mu, alpha1, lmax are set; scale[] and code_len[] are written.
 * Signals are x[offsets[i] .. offsets[i] + lengths[i]). */
fptc_status fptc_train_domain(const float *x, const uint64_t *offsets, const uint64_t *lengths, uint64_t n_signals,
                              double percentile, fptc_domain *domain);

/* The level map of zone 0 (Eq. 2) or 1 (Eq. 3) that fptc_encode_stream
 * applies to an FP64 coefficient, given as its 255 boundaries: bounds[L - 1]
 * (L = 1 .. 255) is the smallest double c whose level is L or more (-inf when
 * every double's is, NaN when none is).  The map is monotone in c, so the
 * level of a non-NaN c, +-inf included, is the number of bounds <= c (NaN:
 * 128).  The GPU
 * encoder settles the bins its FP32 tiers cannot with this table.  bounds
 * must hold 255 doubles; zone must be 0 or 1, else FPTC_ERR_INVALID_ARGUMENT. */
fptc_status fptc_zone_bounds(const fptc_domain *domain, uint32_t zone, double *bounds);

/* Upper bound on the words of a stream of S samples (every word but the last
 * holds at least ceil((65 - lmax) / lmax) codewords). */
uint64_t fptc_word_capacity(const fptc_domain *domain, uint64_t n_samples);

/* Encodes one signal: windows of N (last one zero-padded), Eq. 1 in FP64, keep
 * E bins, three-zone quantizer (Eq. 2, Eq. 3, zone 2 -> 128), canonical Huffman
 * codes packed by Alg. 1.  words / symlen must hold `capacity` entries;
 * *n_words receives the count.  levels (optional) receives the W*E symbols. */
fptc_status fptc_encode_stream(const fptc_domain *domain, const float *x, uint64_t n_samples, uint64_t *words,
                               uint8_t *symlen, uint64_t capacity, uint64_t *n_words, uint8_t *levels);

/* Encodes n signals on n_threads host threads (0 = all cores).  Signal i
 * (x[x_offsets[i] ..], lengths[i] samples, domain domains[domain_idx[i]]) is
 * written to words / symlen at capacity_offsets[i] with room for
 * fptc_word_capacity() words; n_words[i] receives its count. */
fptc_status fptc_encode_batch(const fptc_domain *domains, uint32_t n_domains, const float *x,
                              const uint64_t *x_offsets, const uint64_t *lengths, const uint32_t *domain_idx,
                              uint64_t n, uint64_t *words, uint8_t *symlen, const uint64_t *capacity_offsets,
                              uint64_t *n_words, int n_threads);

#ifdef __cplusplus
}
#endif
#endif /* FPTC_CODEC_H_ */
