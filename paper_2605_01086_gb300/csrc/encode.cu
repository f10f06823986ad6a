// The FPTC encoder on the GPU (include/fptc_encoder.h): Eq. 1, the three-zone
// quantizer of Sec. 3.2 and the SymLen packing of Alg. 1 for many streams.
//
//   k_enc_levels  one thread per window: the zero-padded window's first E
//                 DCT-II bins in FP64 (products and sums rounded separately, in
//                 sample order, then scaled by 2/N, as the host encoder does),
//                 then the zone quantizer of each bin -> level bytes.
//   k_enc_pack    one thread per stream: Alg. 1 over its levels (greedy: a
//                 codeword that does not fit closes the word and starts the
//                 next), words and symbol counts into the stream's room.
// The packing is sequential within a stream, as Alg. 1 is; streams run in
// parallel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fptc_codec.h"
#include "fptc_encoder.h"
#include "fptc_internal.h"
#include "host_util.h"

namespace fptc {
namespace {

struct EncDomain {
  uint32_t N, E, B1, B2;
  double A0, A1, mu, alpha1, log1pmu;
  uint32_t cos_off;   // first double of the E x N cosine table
  uint32_t code_off;  // first entry of the 256 codewords / lengths
};

struct EncSeg {
  uint64_t in_offset;   // first sample in d_x
  uint64_t n_samples;
  uint64_t word_offset;
  uint64_t room;
  uint64_t level_offset;
  uint64_t win_base;    // first global window
  uint64_t n_windows;
  uint32_t domain;
  uint32_t pad;
};

struct EncStatus {
  unsigned int flags;
  unsigned int pad;
  unsigned long long first_bad;
};

struct EncParams {
  const float *x;
  uint64_t *words;
  uint8_t *symlen;
  uint64_t *n_words;
  uint8_t *levels;
  const EncSeg *segs;
  const EncDomain *doms;
  const double *cosv;
  const uint32_t *codes;
  const uint8_t *lens;
  EncStatus *status;
  uint64_t n_segs;
  uint64_t n_windows;
};

__device__ __forceinline__ void enc_flag(EncStatus *st, unsigned int f, uint64_t seg) {
  atomicOr(&st->flags, f);
  atomicMin(&st->first_bad, (unsigned long long)seg);
}

// Eq. 2 with the level map 128 + round(127 q) / 128 - round(128 q), |c| clamped to A0.
__device__ __forceinline__ uint32_t zone0_level(double c, const EncDomain &d) {
  if (!(d.A0 > 1e-30) || isnan(c)) return 128u;
  const double a = fmin(fabs(c), d.A0);
  const double q = log1p(__dmul_rn(d.mu, a / d.A0)) / d.log1pmu;
  long long v = c >= 0.0 ? 128 + (long long)floor(__dadd_rn(__dmul_rn(127.0, q), 0.5))
                         : 128 - (long long)floor(__dadd_rn(__dmul_rn(128.0, q), 0.5));
  return (uint32_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}

// Eq. 3, |c| clamped to A1, deadzone d1 = alpha1 A1.
__device__ __forceinline__ uint32_t zone1_level(double c, const EncDomain &d) {
  if (!(d.A1 > 1e-30) || isnan(c)) return 128u;
  const double d1 = __dmul_rn(d.alpha1, d.A1);
  const double m = fmin(fabs(c), d.A1);
  if (m <= d1) return 128u;
  const double r = __dsub_rn(m, d1) / __dsub_rn(d.A1, d1);
  long long v = c > 0 ? 129 + (long long)floor(__dadd_rn(__dmul_rn(r, 126.0), 0.5))
                      : 127 - (long long)floor(__dadd_rn(__dmul_rn(r, 127.0), 0.5));
  return (uint32_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}

// Segment (caller order) owning global window g.
__device__ __forceinline__ uint64_t enc_segment(const EncSeg *segs, uint64_t n, uint64_t g) {
  uint64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (segs[mid].win_base <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_enc_levels(EncParams p) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= p.n_windows) return;
  const uint64_t s = enc_segment(p.segs, p.n_segs, g);
  const EncSeg sg = p.segs[s];
  const EncDomain d = p.doms[sg.domain];
  const uint64_t w = g - sg.win_base;
  const uint64_t i0 = w * d.N;
  const uint64_t avail = sg.n_samples - i0;  // >= 1
  double xw[128];
  for (uint32_t n = 0; n < d.N; ++n) xw[n] = n < avail ? (double)p.x[sg.in_offset + i0 + n] : 0.0;
  uint8_t *const lv = p.levels + sg.level_offset + w * d.E;
  const double *cw = p.cosv + d.cos_off;
  const double scale = 2.0 / (double)d.N;
  for (uint32_t k = 0; k < d.E; ++k) {
    uint32_t L = 128u;
    if (k < d.B2) {
      const double *row = cw + (size_t)k * d.N;
      double acc = 0.0;
      for (uint32_t n = 0; n < d.N; ++n) acc = __dadd_rn(acc, __dmul_rn(xw[n], row[n]));
      const double c = __dmul_rn(acc, scale);
      L = k < d.B1 ? zone0_level(c, d) : zone1_level(c, d);
    }
    lv[k] = (uint8_t)L;
  }
}

__global__ void __launch_bounds__(128) k_enc_pack(EncParams p) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.n_segs) return;
  const EncSeg sg = p.segs[s];
  const EncDomain d = p.doms[sg.domain];
  const uint8_t *lv = p.levels + sg.level_offset;
  const uint64_t L = sg.n_windows * d.E;
  const uint32_t *code = p.codes + d.code_off;
  const uint8_t *len = p.lens + d.code_off;
  uint64_t *const out = p.words + sg.word_offset;
  uint8_t *const sl = p.symlen + sg.word_offset;
  uint64_t buffer = 0, w = 0;
  uint32_t bits = 0, count = 0;
  bool bad = false;
  for (uint64_t i = 0; i < L; ++i) {
    const uint32_t sym = lv[i];
    const uint32_t cl = __ldg(len + sym);
    if (cl == 0) {
      enc_flag(p.status, FPTC_ENC_FLAG_NO_CODE, s);
      bad = true;
      break;
    }
    if (bits + cl > 64) {  // the codeword does not fit: close the word, retry it on the next
      if (w >= sg.room) {
        enc_flag(p.status, FPTC_ENC_FLAG_ROOM, s);
        bad = true;
        break;
      }
      out[w] = buffer;
      sl[w] = (uint8_t)count;
      ++w;
      buffer = 0;
      bits = 0;
      count = 0;
    }
    buffer |= (uint64_t)__ldg(code + sym) << (64 - bits - cl);
    bits += cl;
    ++count;
  }
  if (!bad && count > 0) {
    if (w >= sg.room) {
      enc_flag(p.status, FPTC_ENC_FLAG_ROOM, s);
    } else {
      out[w] = buffer;
      sl[w] = (uint8_t)count;
      ++w;
    }
  }
  p.n_words[s] = w;
}

struct DevGuard {
  int prev = -1;
  bool ok = true;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

fptc_status enc_cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FPTC_ERR_OUT_OF_MEMORY : FPTC_ERR_CUDA;
}

}  // namespace
}  // namespace fptc

using namespace fptc;

struct fptc_encoder {
  int device = 0;
  uint64_t n_segs = 0, n_windows = 0, n_levels = 0;
  std::vector<uint64_t> level_off;  // caller order
  EncSeg *d_segs = nullptr;
  EncDomain *d_doms = nullptr;
  double *d_cos = nullptr;
  uint32_t *d_codes = nullptr;
  uint8_t *d_lens = nullptr;
  EncStatus *d_status = nullptr;
  uint8_t *d_lev_scratch = nullptr;
};

namespace {

void enc_free(fptc_encoder *e) {
  cudaFree(e->d_segs);
  cudaFree(e->d_doms);
  cudaFree(e->d_cos);
  cudaFree(e->d_codes);
  cudaFree(e->d_lens);
  cudaFree(e->d_status);
  cudaFree(e->d_lev_scratch);
}

template <typename T>
cudaError_t enc_upload(T **dst, const T *src, size_t n) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), std::max<size_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess && n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

EncParams enc_params(const fptc_encoder *e, uint64_t *d_words, uint8_t *d_symlen, uint64_t *d_n_words,
                     uint8_t *levels) {
  EncParams p{};
  p.words = d_words;
  p.symlen = d_symlen;
  p.n_words = d_n_words;
  p.levels = levels;
  p.segs = e->d_segs;
  p.doms = e->d_doms;
  p.cosv = e->d_cos;
  p.codes = e->d_codes;
  p.lens = e->d_lens;
  p.status = e->d_status;
  p.n_segs = e->n_segs;
  p.n_windows = e->n_windows;
  return p;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

fptc_status fptc_encoder_create(fptc_encoder **enc, int device, const fptc_domain *domains, uint32_t n_domains,
                                const fptc_segment *segments, uint64_t n_segments) {
  clear_error();
  if (!enc) {
    set_error("NULL encoder pointer");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  *enc = nullptr;
  if (!domains || n_domains == 0 || (n_segments && !segments)) {
    set_error("need at least one domain and a segment array");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  std::vector<EncDomain> doms(n_domains);
  std::vector<double> cosv;
  std::vector<uint32_t> codes;
  std::vector<uint8_t> lens;
  for (uint32_t d = 0; d < n_domains; ++d) {
    const fptc_domain &dm = domains[d];
    fptc_status st = fptc_validate_domain(&dm);
    if (st != FPTC_OK) return st;
    EncDomain &x = doms[d];
    x.N = dm.N;
    x.E = dm.E;
    x.B1 = dm.B1;
    x.B2 = dm.B2;
    x.A0 = dm.scale[0];
    x.A1 = dm.scale[1];
    x.mu = dm.mu;
    x.alpha1 = dm.alpha1;
    x.log1pmu = std::log1p(dm.mu);
    x.cos_off = (uint32_t)cosv.size();
    for (uint32_t k = 0; k < dm.E; ++k)
      for (uint32_t n = 0; n < dm.N; ++n) cosv.push_back(std::cos(M_PI * (2.0 * n + 1.0) * k / (2.0 * dm.N)));
    x.code_off = (uint32_t)codes.size();
    uint32_t c[256];
    st = fptc_canonical_codes(&dm, c);
    if (st != FPTC_OK) return st;
    for (int s = 0; s < 256; ++s) {
      codes.push_back(c[s]);
      lens.push_back(dm.code_len[s]);
    }
  }
  std::vector<EncSeg> segs(n_segments);
  std::vector<uint64_t> level_off(n_segments);
  std::vector<std::pair<uint64_t, uint64_t>> rooms;
  uint64_t win = 0, lv = 0;
  for (uint64_t i = 0; i < n_segments; ++i) {
    const fptc_segment &s = segments[i];
    if (s.domain >= n_domains) {
      set_error("segment %llu: domain %u out of range", (unsigned long long)i, s.domain);
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    const fptc_domain &dm = domains[s.domain];
    EncSeg &e = segs[i];
    e.in_offset = s.out_offset;
    e.n_samples = s.n_samples;
    e.word_offset = s.word_offset;
    e.room = s.n_words;
    e.level_offset = lv;
    e.win_base = win;
    e.n_windows = (s.n_samples + dm.N - 1) / dm.N;
    e.domain = s.domain;
    e.pad = 0;
    level_off[i] = lv;
    win += e.n_windows;
    lv += e.n_windows * dm.E;
    if (s.n_words) rooms.push_back({s.word_offset, s.word_offset + s.n_words});
  }
  std::sort(rooms.begin(), rooms.end());
  for (size_t i = 1; i < rooms.size(); ++i)
    if (rooms[i].first < rooms[i - 1].second) {
      set_error("segment rooms overlap at word %llu", (unsigned long long)rooms[i].first);
      return FPTC_ERR_INVALID_ARGUMENT;
    }
  DevGuard g(device);
  if (!g.ok) return enc_cuda_fail(cudaGetLastError(), "set device");
  fptc_encoder *e = new fptc_encoder;
  e->device = device;
  e->n_segs = n_segments;
  e->n_windows = win;
  e->n_levels = lv;
  e->level_off = level_off;
  cudaError_t err = enc_upload(&e->d_segs, segs.data(), segs.size());
  if (err == cudaSuccess) err = enc_upload(&e->d_doms, doms.data(), doms.size());
  if (err == cudaSuccess) err = enc_upload(&e->d_cos, cosv.data(), cosv.size());
  if (err == cudaSuccess) err = enc_upload(&e->d_codes, codes.data(), codes.size());
  if (err == cudaSuccess) err = enc_upload(&e->d_lens, lens.data(), lens.size());
  if (err == cudaSuccess) {
    const EncStatus s0{0u, 0u, ~0ull};
    err = enc_upload(&e->d_status, &s0, 1);
  }
  if (err != cudaSuccess) {
    enc_free(e);
    delete e;
    return enc_cuda_fail(err, "encoder upload");
  }
  *enc = e;
  return FPTC_OK;
}

void fptc_encoder_destroy(fptc_encoder *enc) {
  if (!enc) return;
  DevGuard g(enc->device);
  cudaDeviceSynchronize();
  enc_free(enc);
  delete enc;
}

uint64_t fptc_encoder_levels(const fptc_encoder *enc) { return enc ? enc->n_levels : 0; }

fptc_status fptc_encoder_level_offsets(const fptc_encoder *enc, uint64_t *offsets) {
  clear_error();
  if (!enc || (!offsets && enc->n_segs)) {
    set_error("NULL argument");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  std::copy(enc->level_off.begin(), enc->level_off.end(), offsets);
  return FPTC_OK;
}

// One encode: the level kernel (unless the levels are given) and the packing.
static fptc_status enc_run(fptc_encoder *enc, const float *d_x, bool levels_given, const uint8_t *d_levels_in,
                           uint64_t *d_words, uint8_t *d_symlen, uint64_t *d_n_words, uint8_t *d_levels,
                           fptc_stream stream) {
  clear_error();
  if (!enc) {
    set_error("NULL encoder");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  if (enc->n_segs == 0) return FPTC_OK;
  if (!d_words || !d_symlen || !d_n_words || !aligned(d_words, 8) || !aligned(d_n_words, 8)) {
    set_error("d_words, d_symlen and d_n_words are required (8-byte aligned words and counts)");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  if (levels_given && enc->n_levels && !d_levels_in) {
    set_error("d_levels is required");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  if (!levels_given && enc->n_windows && (!d_x || !aligned(d_x, 4))) {
    set_error("d_x is required (float aligned)");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  DevGuard g(enc->device);
  if (!g.ok) return enc_cuda_fail(cudaGetLastError(), "set device");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint8_t *lev = levels_given ? const_cast<uint8_t *>(d_levels_in) : d_levels;
  if (!lev) {
    if (!enc->d_lev_scratch) {  // first encode without a level buffer: the scratch is the encoder's
      cudaError_t e = cudaMalloc(&enc->d_lev_scratch, std::max<uint64_t>(enc->n_levels, 1));
      if (e != cudaSuccess) return enc_cuda_fail(e, "level scratch");
    }
    lev = enc->d_lev_scratch;
  }
  EncParams p = enc_params(enc, d_words, d_symlen, d_n_words, lev);
  p.x = d_x;
  cudaError_t e = cudaSuccess;
  if (!levels_given && enc->n_windows) {
    const uint64_t blocks = (enc->n_windows + 255) / 256;
    k_enc_levels<<<(unsigned)blocks, 256, 0, s>>>(p);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_enc_pack<<<(unsigned)((enc->n_segs + 127) / 128), 128, 0, s>>>(p);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return enc_cuda_fail(e, "encode launch");
  return FPTC_OK;
}

fptc_status fptc_encode_device(fptc_encoder *enc, const float *d_x, uint64_t *d_words, uint8_t *d_symlen,
                               uint64_t *d_n_words, uint8_t *d_levels, fptc_stream stream) {
  return enc_run(enc, d_x, false, nullptr, d_words, d_symlen, d_n_words, d_levels, stream);
}

fptc_status fptc_pack_device(fptc_encoder *enc, const uint8_t *d_levels, uint64_t *d_words, uint8_t *d_symlen,
                             uint64_t *d_n_words, fptc_stream stream) {
  return enc_run(enc, nullptr, true, d_levels, d_words, d_symlen, d_n_words, nullptr, stream);
}

fptc_status fptc_encoder_status(fptc_encoder *enc, uint32_t *flags, uint64_t *first_bad) {
  clear_error();
  if (!enc) {
    set_error("NULL encoder");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  DevGuard g(enc->device);
  cudaError_t e = cudaDeviceSynchronize();
  EncStatus h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, enc->d_status, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    const EncStatus s0{0u, 0u, ~0ull};
    e = cudaMemcpy(enc->d_status, &s0, sizeof(s0), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return enc_cuda_fail(e, "read encoder status");
  if (flags) *flags = h.flags;
  if (first_bad) *first_bad = h.flags ? (uint64_t)h.first_bad : UINT64_MAX;
  if (h.flags) {
    set_error("encoder flagged segment %llu (flags 0x%x)", (unsigned long long)h.first_bad, h.flags);
    return FPTC_ERR_CORRUPT_STREAM;
  }
  return FPTC_OK;
}

}  // extern "C"
