/*
 * fptc_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, FP64 CPU restatement of the FPTC codec ("FPTC: A Fast Parallel
 * Transform-based Codec for Efficient Asymmetric Signal Compression",
 * arXiv 2605.01086): the sequential encoder (Sec. 3.1-3.3, Sec. 4.1, Alg. 1) and
 * a deliberately different decoder (bit-serial canonical Huffman, no lookup
 * table; FP64 inverse transform).  The CUDA decoder is checked against it; it shares
 * no code with it.  Only tests/, __graft_entry__.smoke() and the benchmark's CPU
 * baseline may load it.
 *
 * Readings of the paper taken where it is silent (each also listed in the design
 * notes):
 *  - inverse transform: the exact inverse of Eq. 1, x[n] = C[0]/2 +
 *    sum_{k=1}^{E-1} C[k] cos(pi/N (n+1/2) k); bins k >= E are zero (Sec. 3.1).
 *  - the last, partial window is zero-padded to N when encoding; the decoder
 *    writes only the S real samples.
 *  - zone-0 level map (Eq. 2 gives only q in [0,1]): c >= 0 -> 128 + floor(127 q + 1/2),
 *    c < 0 -> 128 - floor(128 q + 1/2); expander |c| = (A0/mu)((1+mu)^q - 1).
 *  - zone-1 reconstruction at the lattice points of Eq. 3:
 *    L >= 129 -> d1 + (L-129)/126 (A1-d1), L <= 127 -> -(d1 + (127-L)/127 (A1-d1)).
 *  - |c| is clamped to A_z before quantizing; a zone with A_z <= 1e-30 maps
 *    everything to 128 and dequantizes to 0.
 *  - rounding is floor(x + 1/2) in FP64.
 *  - A_z is one scale per zone: the nearest-rank percentile of |c| pooled over
 *    all training windows and all bins of the zone.
 *  - the symbol histogram gets +1 on every one of the 256 counts, so every
 *    level has a code.
 *  - canonical codes are assigned in (length, symbol) order, shortest first,
 *    starting from code 0 (the DEFLATE convention).
 *  - symbols are stored window-major; codewords MSB-first in each 64-bit word
 *    (Alg. 1, shift = 64 - bit_size - code_len).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_NOCODE -2
#define OR_ERR_CAPACITY -3
#define OR_ERR_OVERRUN -4
#define OR_ERR_INVALID_CODE -5
#define OR_ERR_COUNT -6
#define OR_ERR_NOMEM -7

typedef struct {
  int32_t N, E, B1, B2;
  double mu, alpha1;
  double A[3];
  int32_t lmax;
  uint8_t code_len[256];
} or_domain;

/* ---- Sec. 3.1, Eq. 1: windowed DCT-II and its inverse -------------------- */

/* cos(pi/N (n + 1/2) k), the kernel of Eq. 1 */
double or_basis(int32_t N, int32_t n, int32_t k) {
  return cos(M_PI / (double)N * ((double)n + 0.5) * (double)k);
}

/* Eq. 1 for one window of N samples, keeping the first E coefficients (Sec. 3.1). */
void or_dct2(const double *x, int32_t N, int32_t E, double *C) {
  for (int32_t k = 0; k < E; ++k) {
    double s = 0.0;
    for (int32_t n = 0; n < N; ++n) s += x[n] * or_basis(N, n, k);
    C[k] = 2.0 / (double)N * s;
  }
}

/* Inverse of Eq. 1 with bins k >= E taken as zero. */
void or_idct3(const double *C, int32_t E, int32_t N, double *x) {
  for (int32_t n = 0; n < N; ++n) {
    double s = E > 0 ? C[0] / 2.0 : 0.0;
    for (int32_t k = 1; k < E; ++k) s += C[k] * or_basis(N, n, k);
    x[n] = s;
  }
}

/* Same two transforms with a precomputed table tab[k*N + n] = or_basis(N, n, k). */
static void dct2_tab(const double *x, int32_t N, int32_t E, const double *tab, double *C) {
  for (int32_t k = 0; k < E; ++k) {
    double s = 0.0;
    for (int32_t n = 0; n < N; ++n) s += x[n] * tab[(size_t)k * N + n];
    C[k] = 2.0 / (double)N * s;
  }
}

static void idct3_tab(const double *C, int32_t E, int32_t N, const double *tab, double *x) {
  for (int32_t n = 0; n < N; ++n) {
    double s = E > 0 ? C[0] / 2.0 : 0.0;
    for (int32_t k = 1; k < E; ++k) s += C[k] * tab[(size_t)k * N + n];
    x[n] = s;
  }
}

static double *basis_table(int32_t N, int32_t E) {
  double *tab = (double *)malloc(sizeof(double) * (size_t)N * (size_t)(E > 0 ? E : 1));
  if (!tab) return NULL;
  for (int32_t k = 0; k < E; ++k)
    for (int32_t n = 0; n < N; ++n) tab[(size_t)k * N + n] = or_basis(N, n, k);
  return tab;
}

/* ---- Sec. 3.2: hybrid three-zone quantizer -------------------------------- */

/* zone 0 = [0, B1), zone 1 = [B1, B2), zone 2 = [B2, E) */
int32_t or_zone(const or_domain *d, int32_t k) { return k < d->B1 ? 0 : (k < d->B2 ? 1 : 2); }

/* Eq. 2 (mu-law companding) with the 8-bit level map of Sec. 3.2.1. */
static int32_t quantize_zone0(double c, double A, double mu) {
  if (!(A > 1e-30) || isnan(c)) return 128;
  double a = fabs(c);
  if (a > A) a = A;
  double q = log(1.0 + mu * a / A) / log(1.0 + mu);
  int32_t L;
  if (c >= 0.0)
    L = 128 + (int32_t)floor(q * 127.0 + 0.5);
  else
    L = 128 - (int32_t)floor(q * 128.0 + 0.5);
  if (L < 0) L = 0;
  if (L > 255) L = 255;
  return L;
}

/* Eq. 3 (linear deadzone), |c| clamped to A1. */
static int32_t quantize_zone1(double c, double A, double alpha) {
  if (!(A > 1e-30) || isnan(c)) return 128;
  double d1 = alpha * A;
  double span = A - d1;
  double cc = c;
  if (cc > A) cc = A;
  if (cc < -A) cc = -A;
  int32_t L = 128;
  if (cc > d1)
    L = 129 + (int32_t)floor((cc - d1) / span * 126.0 + 0.5);
  else if (cc < -d1)
    L = 127 - (int32_t)floor((fabs(cc) - d1) / span * 127.0 + 0.5);
  if (L < 0) L = 0;
  if (L > 255) L = 255;
  return L;
}

int32_t or_quantize(const or_domain *d, int32_t zone, double c) {
  switch (zone) {
    case 0: return quantize_zone0(c, d->A[0], d->mu);
    case 1: return quantize_zone1(c, d->A[1], d->alpha1);
    default: return 128; /* Sec. 3.2.3: zone 2 maps every coefficient to the zero bin */
  }
}

/* Inverse of the zone maps with scale A (the expander / lattice reconstruction). */
static double dequantize_with(int32_t zone, int32_t L, double A, double mu, double alpha) {
  if (zone >= 2 || L == 128 || !(A > 1e-30)) return 0.0;
  if (zone == 0) {
    double q = L > 128 ? (double)(L - 128) / 127.0 : (double)(128 - L) / 128.0;
    double m = A / mu * (pow(1.0 + mu, q) - 1.0);
    return L > 128 ? m : -m;
  }
  double d1 = alpha * A;
  double span = A - d1;
  if (L >= 129) return d1 + (double)(L - 129) / 126.0 * span;
  return -(d1 + (double)(127 - L) / 127.0 * span);
}

double or_dequantize(const or_domain *d, int32_t zone, int32_t L) {
  double A = zone < 2 ? d->A[zone] : 0.0;
  return dequantize_with(zone, L, A, d->mu, d->alpha1);
}

/* d c_hat / d A_z: both zone maps are linear in A_z, so this is the
 * reconstruction at A_z = 1 (zero when the zone is switched off). */
double or_dequantize_unit(const or_domain *d, int32_t zone, int32_t L) {
  if (zone >= 2 || !(d->A[zone] > 1e-30)) return 0.0;
  return dequantize_with(zone, L, 1.0, d->mu, d->alpha1);
}

/* ---- Sec. 3.2.1: per-zone scale as a clipped (nearest-rank) percentile ---- */

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Sorts v in place; returns the value of nearest rank ceil(p/100 * n).  The rank
 * is taken with a 1e-9 slack so that a decimal percentile such as 99.9, which
 * is not exact in binary, lands on its exact rank (99.9% of 1000 -> rank 999). */
double or_percentile(double *v, uint64_t n, double p) {
  if (n == 0) return 0.0;
  qsort(v, (size_t)n, sizeof(double), cmp_double);
  double r = ceil(p / 100.0 * (double)n - 1e-9);
  int64_t idx = (int64_t)r - 1;
  if (idx < 0) idx = 0;
  if (idx > (int64_t)n - 1) idx = (int64_t)n - 1;
  return v[idx];
}

/* ---- Sec. 3.3: length-limited code lengths (package-merge) ---------------- */

typedef struct {
  uint64_t w;
  int32_t sym; /* >= 0 leaf symbol, -1 package */
} pm_item;

/* Larmore-Hirschberg package-merge: optimal code lengths <= lmax for the
 * symbols with freq > 0 (others get length 0).  Lists are kept for every
 * denomination 2^-l, l = lmax..1; list l merges the leaves (sorted by weight,
 * then symbol) with the pairwise packages of list l+1 (a leaf goes first on
 * equal weight).  The first 2n-2 items of list 1 are selected; a selected
 * package at level l selects the two items of level l+1 it was made from, and
 * every selected leaf adds one bit to its symbol's length.
 * Returns 0, or OR_ERR_ARG if 2^lmax < number of used symbols. */
int32_t or_package_merge(const uint64_t *freq, int32_t n_sym, int32_t lmax, uint8_t *len_out) {
  if (n_sym <= 0 || lmax < 1 || lmax > 32) return OR_ERR_ARG;
  for (int32_t i = 0; i < n_sym; ++i) len_out[i] = 0;
  int32_t n = 0;
  for (int32_t i = 0; i < n_sym; ++i) n += freq[i] > 0;
  if (n == 0) return OR_OK;
  if (n == 1) { /* one used symbol: give it a 1-bit code */
    for (int32_t i = 0; i < n_sym; ++i)
      if (freq[i] > 0) len_out[i] = 1;
    return OR_OK;
  }
  if (lmax < 32 && ((uint64_t)1 << lmax) < (uint64_t)n) return OR_ERR_ARG;

  /* sorted leaves: by (weight, symbol) -- insertion sort, n <= n_sym is small */
  pm_item *leaves = (pm_item *)malloc(sizeof(pm_item) * (size_t)n);
  if (!leaves) return OR_ERR_NOMEM;
  int32_t m = 0;
  for (int32_t i = 0; i < n_sym; ++i) {
    if (freq[i] == 0) continue;
    pm_item it = {freq[i], i};
    int32_t j = m;
    while (j > 0 && (leaves[j - 1].w > it.w || (leaves[j - 1].w == it.w && leaves[j - 1].sym > it.sym))) {
      leaves[j] = leaves[j - 1];
      --j;
    }
    leaves[j] = it;
    ++m;
  }

  /* lists[l] for l = 1..lmax; each has at most 2n - 1 items */
  pm_item **lists = (pm_item **)calloc((size_t)lmax + 1, sizeof(pm_item *));
  int32_t *cnt = (int32_t *)calloc((size_t)lmax + 1, sizeof(int32_t));
  if (!lists || !cnt) {
    free(leaves); free(lists); free(cnt);
    return OR_ERR_NOMEM;
  }
  int32_t rc = OR_OK;
  for (int32_t l = lmax; l >= 1; --l) {
    lists[l] = (pm_item *)malloc(sizeof(pm_item) * (size_t)(2 * n));
    if (!lists[l]) { rc = OR_ERR_NOMEM; break; }
    if (l == lmax) {
      memcpy(lists[l], leaves, sizeof(pm_item) * (size_t)n);
      cnt[l] = n;
      continue;
    }
    int32_t np = cnt[l + 1] / 2; /* packages of the level below */
    int32_t a = 0, b = 0, o = 0;
    while (a < n || b < np) {
      uint64_t pw = b < np ? lists[l + 1][2 * b].w + lists[l + 1][2 * b + 1].w : 0;
      if (b >= np || (a < n && leaves[a].w <= pw)) {
        lists[l][o++] = leaves[a++];
      } else {
        pm_item p = {pw, -1};
        lists[l][o++] = p;
        ++b;
      }
    }
    cnt[l] = o;
  }
  if (rc == OR_OK) {
    int32_t take = 2 * n - 2;
    for (int32_t l = 1; l <= lmax && take > 0; ++l) {
      if (take > cnt[l]) { rc = OR_ERR_ARG; break; }
      int32_t packages = 0;
      for (int32_t i = 0; i < take; ++i) {
        if (lists[l][i].sym >= 0)
          len_out[lists[l][i].sym] += 1;
        else
          ++packages;
      }
      take = 2 * packages;
    }
  }
  for (int32_t l = 1; l <= lmax; ++l) free(lists[l]);
  free(lists);
  free(cnt);
  free(leaves);
  return rc;
}

/* Canonical codewords from lengths ("canonized", Sec. 3.3): codes of one length
 * are consecutive, shorter lengths first, symbols in increasing order.
 * Returns OR_ERR_ARG if the lengths break the Kraft inequality. */
int32_t or_canonical_codes(const uint8_t *len, int32_t n_sym, int32_t lmax, uint32_t *code_out) {
  uint64_t bl_count[33] = {0};
  uint64_t next[33] = {0};
  for (int32_t i = 0; i < n_sym; ++i) {
    if (len[i] > lmax || len[i] > 32) return OR_ERR_ARG;
    bl_count[len[i]]++;
  }
  bl_count[0] = 0;
  /* Kraft: sum 2^(lmax - len) <= 2^lmax */
  uint64_t kraft = 0;
  for (int32_t b = 1; b <= lmax; ++b) kraft += bl_count[b] << (lmax - b);
  if (kraft > ((uint64_t)1 << lmax)) return OR_ERR_ARG;
  uint64_t c = 0;
  for (int32_t b = 1; b <= lmax; ++b) {
    c = (c + bl_count[b - 1]) << 1;
    next[b] = c;
  }
  for (int32_t i = 0; i < n_sym; ++i) {
    code_out[i] = 0;
    if (len[i]) code_out[i] = (uint32_t)next[len[i]]++;
  }
  return OR_OK;
}

/* ---- Sec. 4.1, Alg. 1: SymLen packing ------------------------------------ */

/* Greedy packing of whole codewords, MSB first, into 64-bit words; symlen[w]
 * is the number of codewords in word w.  Returns the number of words, or a
 * negative error. */
int64_t or_pack_symlen(const uint8_t *X, uint64_t L, const uint32_t *code, const uint8_t *len,
                       uint64_t *out, uint8_t *symlen, uint64_t capacity) {
  uint64_t i = 0, w = 0, buffer = 0;
  uint32_t bit_size = 0, count = 0;
  while (i < L) {
    uint32_t cl = len[X[i]];
    uint64_t cw = code[X[i]];
    if (cl == 0) return OR_ERR_NOCODE;
    if (cl > 64) return OR_ERR_ARG;
    if (bit_size + cl > 64) {
      if (w >= capacity) return OR_ERR_CAPACITY;
      out[w] = buffer;
      symlen[w] = (uint8_t)count;
      ++w;
      buffer = 0;
      bit_size = 0;
      count = 0;
      /* the same symbol is retried on the next word */
    } else {
      uint32_t shift = 64 - bit_size - cl;
      buffer |= cw << shift;
      bit_size += cl;
      ++count;
      ++i;
    }
  }
  if (count > 0) {
    if (w >= capacity) return OR_ERR_CAPACITY;
    out[w] = buffer;
    symlen[w] = (uint8_t)count;
    ++w;
  }
  return (int64_t)w;
}

/* Bit-serial canonical decode (no lookup table): for each word, decode exactly
 * symlen[w] codewords reading one bit at a time, MSB first.  Returns 0 and
 * fills X[0..L), or a negative error (bit overrun, invalid code, count). */
int32_t or_unpack_symlen(const uint64_t *words, const uint8_t *symlen, uint64_t n_words, const uint8_t *len,
                         int32_t lmax, uint8_t *X, uint64_t L) {
  if (lmax < 1 || lmax > 32) return OR_ERR_ARG;
  uint64_t count[33] = {0}, first[33] = {0}, base[33] = {0};
  uint8_t sorted[256];
  for (int32_t i = 0; i < 256; ++i) {
    if (len[i] > lmax) return OR_ERR_ARG;
    count[len[i]]++;
  }
  count[0] = 0;
  uint64_t c = 0, b = 0;
  for (int32_t l = 1; l <= lmax; ++l) {
    c = (c + count[l - 1]) << 1;
    first[l] = c;
    base[l] = b;
    b += count[l];
  }
  int32_t o = 0;
  for (int32_t l = 1; l <= lmax; ++l)
    for (int32_t s = 0; s < 256; ++s)
      if (len[s] == l) sorted[o++] = (uint8_t)s;

  uint64_t out = 0;
  for (uint64_t w = 0; w < n_words; ++w) {
    uint64_t word = words[w];
    uint32_t pos = 0;
    for (uint32_t j = 0; j < symlen[w]; ++j) {
      uint64_t cv = 0;
      int found = -1;
      for (int32_t l = 1; l <= lmax; ++l) {
        if (pos >= 64) return OR_ERR_OVERRUN;
        cv = (cv << 1) | ((word >> (63 - pos)) & 1u);
        ++pos;
        if (count[l] && cv >= first[l] && cv - first[l] < count[l]) {
          found = sorted[base[l] + (cv - first[l])];
          break;
        }
      }
      if (found < 0) return OR_ERR_INVALID_CODE;
      if (out >= L) return OR_ERR_COUNT;
      X[out++] = (uint8_t)found;
    }
  }
  return out == L ? OR_OK : OR_ERR_COUNT;
}

/* ---- whole streams --------------------------------------------------------- */

static uint64_t n_windows(uint64_t S, int32_t N) { return (S + (uint64_t)N - 1) / (uint64_t)N; }

/* Quantized symbol stream of one signal: window (zero-padded), Eq. 1, keep E,
 * per-bin zone quantizer; window-major. */
int32_t or_quantize_stream(const float *x, uint64_t S, const or_domain *d, uint8_t *levels) {
  const int32_t N = d->N, E = d->E;
  double *tab = basis_table(N, E);
  double *xw = (double *)malloc(sizeof(double) * (size_t)N);
  double *C = (double *)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
  if (!tab || !xw || !C) {
    free(tab); free(xw); free(C);
    return OR_ERR_NOMEM;
  }
  uint64_t W = n_windows(S, N);
  for (uint64_t w = 0; w < W; ++w) {
    for (int32_t n = 0; n < N; ++n) {
      uint64_t i = w * (uint64_t)N + (uint64_t)n;
      xw[n] = i < S ? (double)x[i] : 0.0;
    }
    dct2_tab(xw, N, E, tab, C);
    for (int32_t k = 0; k < E; ++k) levels[w * (uint64_t)E + k] = (uint8_t)or_quantize(d, or_zone(d, k), C[k]);
  }
  free(tab); free(xw); free(C);
  return OR_OK;
}

/* Encoder of Fig. 5: transform, quantize, Huffman + SymLen (Alg. 1). */
int32_t or_encode_stream(const float *x, uint64_t S, const or_domain *d, uint64_t *words, uint8_t *symlen,
                         uint64_t capacity, uint64_t *n_words_out, uint8_t *levels_out) {
  uint64_t L = n_windows(S, d->N) * (uint64_t)d->E;
  uint8_t *X = levels_out ? levels_out : (uint8_t *)malloc(L ? L : 1);
  if (!X) return OR_ERR_NOMEM;
  int32_t rc = or_quantize_stream(x, S, d, X);
  uint32_t code[256];
  if (rc == OR_OK) rc = or_canonical_codes(d->code_len, 256, d->lmax, code);
  if (rc == OR_OK) {
    int64_t nw = or_pack_symlen(X, L, code, d->code_len, words, symlen, capacity);
    if (nw < 0)
      rc = (int32_t)nw;
    else
      *n_words_out = (uint64_t)nw;
  }
  if (!levels_out) free(X);
  return rc;
}

/* Levels -> samples: dequantize (zone inverse), inverse of Eq. 1, reassemble
 * windows and drop the padding past S. */
int32_t or_reconstruct(const uint8_t *levels, uint64_t S, const or_domain *d, double *x_out) {
  const int32_t N = d->N, E = d->E;
  double *tab = basis_table(N, E);
  double *xw = (double *)malloc(sizeof(double) * (size_t)N);
  double *C = (double *)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
  if (!tab || !xw || !C) {
    free(tab); free(xw); free(C);
    return OR_ERR_NOMEM;
  }
  uint64_t W = n_windows(S, N);
  for (uint64_t w = 0; w < W; ++w) {
    for (int32_t k = 0; k < E; ++k) C[k] = or_dequantize(d, or_zone(d, k), levels[w * (uint64_t)E + k]);
    idct3_tab(C, E, N, tab, xw);
    for (int32_t n = 0; n < N; ++n) {
      uint64_t i = w * (uint64_t)N + (uint64_t)n;
      if (i < S) x_out[i] = xw[n];
    }
  }
  free(tab); free(xw); free(C);
  return OR_OK;
}

/* Decoder: bit-serial Huffman, then reconstruction. levels_out is optional. */
int32_t or_decode_stream(const uint64_t *words, const uint8_t *symlen, uint64_t n_words, uint64_t S,
                         const or_domain *d, double *x_out, uint8_t *levels_out) {
  uint64_t L = n_windows(S, d->N) * (uint64_t)d->E;
  uint8_t *X = levels_out ? levels_out : (uint8_t *)malloc(L ? L : 1);
  if (!X) return OR_ERR_NOMEM;
  int32_t rc = or_unpack_symlen(words, symlen, n_words, d->code_len, d->lmax, X, L);
  if (rc == OR_OK && x_out) rc = or_reconstruct(X, S, d, x_out);
  if (!levels_out) free(X);
  return rc;
}

/* Adjoint of the reconstruction for a loss with gradient g_x (length S) on the
 * samples: g_C[w,k] = sum_n g_x[wN+n] * dx[n]/dC[k] (1/2 for k = 0, the Eq. 1
 * kernel otherwise; samples past S contribute nothing), and
 * grad_A[z] += sum over bins of zone z of g_C * d c_hat/d A_z.
 * g_C (W*E) is optional. */
int32_t or_backward_stream(const uint8_t *levels, uint64_t S, const or_domain *d, const double *g_x, double *g_C,
                           double *grad_A) {
  const int32_t N = d->N, E = d->E;
  double *tab = basis_table(N, E);
  if (!tab) return OR_ERR_NOMEM;
  uint64_t W = n_windows(S, N);
  for (uint64_t w = 0; w < W; ++w) {
    for (int32_t k = 0; k < E; ++k) {
      double s = 0.0;
      for (int32_t n = 0; n < N; ++n) {
        uint64_t i = w * (uint64_t)N + (uint64_t)n;
        double g = i < S ? g_x[i] : 0.0;
        s += g * (k == 0 ? 0.5 : tab[(size_t)k * N + n]);
      }
      if (g_C) g_C[w * (uint64_t)E + k] = s;
      int32_t z = or_zone(d, k);
      if (z < 2) grad_A[z] += s * or_dequantize_unit(d, z, levels[w * (uint64_t)E + k]);
    }
  }
  free(tab);
  return OR_OK;
}

/* ---- Sec. 3.3 / Fig. 4: per-domain prebuilt structures -------------------- */

/* Trains A_0, A_1 (percentile of |c| per zone) and the code lengths (histogram
 * of the quantized training coefficients, +1 smoothing, package-merge) for a
 * domain whose N, E, B1, B2, mu, alpha1, lmax are set.  Signals are given as
 * one flat array with offsets and lengths. */
int32_t or_train_domain(const float *x, const uint64_t *offsets, const uint64_t *lengths, int32_t n_signals,
                        double percentile, or_domain *d) {
  const int32_t N = d->N, E = d->E;
  if (N < 1 || E < 1 || E > N || d->B1 < 0 || d->B1 > d->B2 || d->B2 > E) return OR_ERR_ARG;
  uint64_t total_w = 0;
  for (int32_t s = 0; s < n_signals; ++s) total_w += n_windows(lengths[s], N);
  double *coef = (double *)malloc(sizeof(double) * (size_t)(total_w * (uint64_t)E + 1));
  double *tab = basis_table(N, E);
  double *xw = (double *)malloc(sizeof(double) * (size_t)N);
  if (!coef || !tab || !xw) {
    free(coef); free(tab); free(xw);
    return OR_ERR_NOMEM;
  }
  uint64_t row = 0;
  for (int32_t s = 0; s < n_signals; ++s) {
    const float *xs = x + offsets[s];
    uint64_t W = n_windows(lengths[s], N);
    for (uint64_t w = 0; w < W; ++w, ++row) {
      for (int32_t n = 0; n < N; ++n) {
        uint64_t i = w * (uint64_t)N + (uint64_t)n;
        xw[n] = i < lengths[s] ? (double)xs[i] : 0.0;
      }
      dct2_tab(xw, N, E, tab, coef + row * (uint64_t)E);
    }
  }
  /* per-zone percentile of |c| */
  for (int32_t z = 0; z < 2; ++z) {
    int32_t k0 = z == 0 ? 0 : d->B1, k1 = z == 0 ? d->B1 : d->B2;
    uint64_t m = total_w * (uint64_t)(k1 - k0);
    double *v = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    if (!v) {
      free(coef); free(tab); free(xw);
      return OR_ERR_NOMEM;
    }
    uint64_t o = 0;
    for (uint64_t r = 0; r < total_w; ++r)
      for (int32_t k = k0; k < k1; ++k) v[o++] = fabs(coef[r * (uint64_t)E + k]);
    d->A[z] = or_percentile(v, m, percentile);
    free(v);
  }
  d->A[2] = 0.0;
  /* histogram of levels, +1 smoothing, package-merge */
  uint64_t hist[256];
  for (int32_t i = 0; i < 256; ++i) hist[i] = 1;
  for (uint64_t r = 0; r < total_w; ++r)
    for (int32_t k = 0; k < E; ++k) hist[or_quantize(d, or_zone(d, k), coef[r * (uint64_t)E + k])]++;
  int32_t rc = or_package_merge(hist, 256, d->lmax, d->code_len);
  free(coef); free(tab); free(xw);
  return rc;
}

/* ---- batches (OpenMP over independent streams) ----------------------------- */

/* Encodes stream i of a batch into words + cap_off[i] (capacity cap[i]). */
int32_t or_encode_many(const float *x, const uint64_t *x_off, const uint64_t *S, const int32_t *dom,
                       const or_domain *domains, uint64_t count, uint64_t *words, uint8_t *symlen,
                       const uint64_t *cap_off, const uint64_t *cap, uint64_t *n_words, int32_t n_threads) {
  int32_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1) reduction(| : bad)
  for (int64_t i = 0; i < (int64_t)count; ++i) {
    int32_t rc = or_encode_stream(x + x_off[i], S[i], &domains[dom[i]], words + cap_off[i], symlen + cap_off[i],
                                  cap[i], &n_words[i], NULL);
    if (rc != OR_OK) bad |= 1;
  }
  return bad ? OR_ERR_ARG : OR_OK;
}

/* Decodes stream i into x_out + out_off[i] (FP64); levels optional at lv_off[i]. */
int32_t or_decode_many(const uint64_t *words, const uint8_t *symlen, const uint64_t *w_off, const uint64_t *n_words,
                       const uint64_t *S, const int32_t *dom, const or_domain *domains, uint64_t count, double *x_out,
                       const uint64_t *out_off, uint8_t *levels, const uint64_t *lv_off, int32_t n_threads) {
  int32_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1) reduction(| : bad)
  for (int64_t i = 0; i < (int64_t)count; ++i) {
    int32_t rc = or_decode_stream(words + w_off[i], symlen + w_off[i], n_words[i], S[i], &domains[dom[i]],
                                  x_out ? x_out + out_off[i] : NULL, levels ? levels + lv_off[i] : NULL);
    if (rc != OR_OK) bad |= 1;
  }
  return bad ? OR_ERR_ARG : OR_OK;
}

/* Size of the struct, so the Python binding can check its mirror. */
uint64_t or_domain_size(void) { return sizeof(or_domain); }
