// The FPTC encoder on the GPU (include/fptc_encoder.h): Eq. 1, the three-zone
// quantizer of Sec. 3.2 and the SymLen packing of Alg. 1 for many streams.
//
//   k_enc_levels  one thread per (window, bin): the DCT-II bin of the
//                 zero-padded window as a compensated FP32 dot product with a
//                 bound on its error, and the zone quantizer.  Every zone map
//                 is monotone in the coefficient, so when the levels at c - err
//                 and c + err agree
//                 the FP64 coefficient (which lies between) has that level too;
//                 otherwise the bin goes to a list that k_enc_fallback computes
//                 again in FP64 (products and sums rounded separately, in
//                 sample order, then scaled by 2/N, as the host encoder does),
//                 one bin per lane, and quantizes from that.
//   k_enc_scan    one thread per stream: Alg. 1's state (word, bits used,
//                 codewords in the word) over the code lengths alone, recorded
//                 at every block of kPackBlock symbols; zeroes the words two
//                 blocks share; the stream's word count, room and code checks.
//   k_enc_pack    one thread per block: Alg. 1 from the recorded state, whole
//                 words with plain stores, the words shared with the previous
//                 or next block with 64-bit atomicOr (their codeword bits are
//                 disjoint), each word's symbol count by the block that closes it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "fptc_codec.h"
#include "fptc_encoder.h"
#include "fptc_internal.h"
#include "host_util.h"

namespace fptc {
namespace {

constexpr uint32_t kPackBlock = 4096;  // symbols per packing block

struct EncDomain {
  uint32_t N, E, B1, B2;
  double A0, A1, mu, alpha1, log1pmu;
  uint32_t cos_off;   // first entry of the E x N cosine tables (FP64 and FP32 copies)
  uint32_t code_off;  // first entry of the 256 codewords / lengths
  // FP32 forms for the fast evaluation of the quantizer
  float A0f, A1f, muf, d1f, inv_A0f, inv_span1f, inv_log1pmuf;
  double d1;             // alpha1 A1 as the FP64 quantizer computes it
  float slack0, slack1;  // per zone: an input width that covers the FP32 evaluation error
};

struct EncSeg {
  uint64_t in_offset;   // first sample in d_x
  uint64_t n_samples;
  uint64_t word_offset;
  uint64_t room;
  uint64_t level_offset;
  uint64_t n_windows;
  uint64_t block_base;  // first global packing block
  uint32_t domain;
  uint32_t pad;
};

// Alg. 1's state before the first symbol of a packing block.
struct PackState {
  uint64_t word;   // word of the stream being filled
  uint32_t bits;   // bits used in it
  uint32_t count;  // codewords in it
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
  const float *cosf;
  const uint32_t *codes;
  const uint8_t *lens;
  PackState *blocks;
  uint32_t *seg_bad;
  unsigned long long *fb_list;   // bins whose level the FP64 coefficient decides
  unsigned int *fb_count;
  uint32_t fb_cap;
  EncStatus *status;
  uint64_t n_segs;
  uint64_t n_levels;
  uint64_t n_blocks;
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

__device__ __forceinline__ uint32_t bin_level(uint32_t k, double c, const EncDomain &d) {
  return k < d.B1 ? zone0_level(c, d) : zone1_level(c, d);
}

// Zone 0's map evaluated in FP32 (reciprocals, log1pf): off from the FP64
// evaluation by less than the zone's slack in the coefficient (both are close
// to the exact monotone map), so used only to bracket it.
__device__ __forceinline__ uint32_t zone0_level32(float c, const EncDomain &d) {
  if (!(d.A0 > 1e-30) || isnan(c)) return 128u;
  const float a = fminf(fabsf(c), d.A0f);
  const float q = log1pf(d.muf * (a * d.inv_A0f)) * d.inv_log1pmuf;
  const int v = c >= 0.0f ? 128 + (int)floorf(fmaf(127.0f, q, 0.5f)) : 128 - (int)floorf(fmaf(128.0f, q, 0.5f));
  return (uint32_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}
// Zone 1 decided from the compensated coefficient: cd (FP64 value of the
// compensated sum, |cd - c64| <= err_d) settles the deadzone test exactly
// unless |cd| is within err_d of d1; outside the deadzone the linear map is
// bracketed in FP32 (a = |c|, bracket half-width m).  Returns false when the
// FP64 coefficient has to decide.
__device__ __forceinline__ bool zone1_decide(float c, double cd, double err_d, float m, const EncDomain &d,
                                             uint32_t &L) {
  if (!(d.A1 > 1e-30) || isnan(c)) {
    L = 128u;
    return true;
  }
  const double ac = fabs(cd);
  if (ac + err_d < d.d1) {
    L = 128u;
    return true;
  }
  if (ac - err_d <= d.d1) return false;  // at the deadzone edge
  const float a = fabsf(c);
  const float k = c > 0.0f ? 126.0f : 127.0f;
  const float r0 = fmaxf((fminf(a - m, d.A1f) - d.d1f) * d.inv_span1f, 0.0f);
  const float r1 = fmaxf((fminf(a + m, d.A1f) - d.d1f) * d.inv_span1f, 0.0f);
  const int v0 = (int)floorf(fmaf(r0, k, 0.5f)), v1 = (int)floorf(fmaf(r1, k, 0.5f));
  if (v0 != v1) return false;
  const int v = c > 0.0f ? 129 + v0 : 127 - v0;
  L = (uint32_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
  return true;
}


// Index i of the last entry with base(i) <= g over n ascending entries.
template <class F>
__device__ __forceinline__ uint64_t last_leq(uint64_t n, uint64_t g, F base) {
  uint64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (base(mid) <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Level of bin g (global level index) from the FP64 coefficient, computed as
// the host encoder does: products and sums rounded separately, in sample order,
// then scaled by 2/N.
__device__ __forceinline__ uint32_t level_fp64(const EncParams &p, uint64_t g) {
  const uint64_t s = last_leq(p.n_segs, g, [&](uint64_t i) { return p.segs[i].level_offset; });
  const EncSeg sg = p.segs[s];
  const EncDomain d = p.doms[sg.domain];
  const uint64_t local = g - sg.level_offset;
  const uint64_t w = local / d.E;
  const uint32_t k = (uint32_t)(local - w * d.E);
  const uint64_t avail = sg.n_samples - w * d.N;
  const float *src = p.x + sg.in_offset + w * d.N;
  const double *row = p.cosv + d.cos_off + (size_t)k * d.N;
  double a64 = 0.0;
  for (uint32_t n = 0; n < d.N; ++n) a64 = __dadd_rn(a64, __dmul_rn(n < avail ? (double)src[n] : 0.0, row[n]));
  return bin_level(k, __dmul_rn(a64, 2.0 / (double)d.N), d);
}

// One thread per (window, bin): thread g writes level g of the level buffer
// (streams in caller order, windows, bins), so a warp covers a few windows, the
// lanes of a window read its samples as broadcasts and the FP32 cosines (a
// high and a low part) are stored transposed (cosf[2 (n E + k)]) for one
// wavefront per sample.  The bin is accumulated as a compensated FP32 dot
// product (exact products by FMA, exact sums by two-sum), whose error is
// O((N u)^2 sum |x|) + u |c|; the quantizer is evaluated in FP32 at the ends
// of a bracket that covers that error and the FP32 evaluation's own slack.
// Bins whose bracket straddles a level boundary go to a list for
// k_enc_fallback (or, when the list is full, are decided here in FP64).
__global__ void __launch_bounds__(256) k_enc_levels(EncParams p) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= p.n_levels) return;
  const uint64_t s = last_leq(p.n_segs, g, [&](uint64_t i) { return p.segs[i].level_offset; });
  const EncSeg sg = p.segs[s];
  const EncDomain d = p.doms[sg.domain];
  const uint32_t N = d.N, E = d.E;
  const uint64_t local = g - sg.level_offset;
  const uint64_t w = local / E;
  const uint32_t k = (uint32_t)(local - w * E);
  uint32_t L = 128u;
  if (k < d.B2) {
    const uint64_t i0 = w * N;
    const uint64_t avail = sg.n_samples - i0;  // >= 1
    const uint32_t nn = avail < N ? (uint32_t)avail : N;  // samples past S are zero
    const float *src = p.x + sg.in_offset + i0;
    const float2 *ct = reinterpret_cast<const float2 *>(p.cosf) + d.cos_off + k;
    float hi = 0.0f, lo = 0.0f, s1 = 0.0f;
    for (uint32_t n = 0; n < nn; ++n) {
      const float xv = src[n];
      const float2 cs = ct[(size_t)n * E];
      // explicit roundings (no contraction): the exact product error by FMA, an exact two-sum
      const float pr = __fmul_rn(xv, cs.x);
      const float pe = __fadd_rn(__fmaf_rn(xv, cs.x, -pr), __fmul_rn(xv, cs.y));
      const float t = __fadd_rn(hi, pr);
      const float bp = __fsub_rn(t, hi);
      lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(pr, bp)), pe));
      hi = t;
      s1 += fabsf(xv);
    }
    const float c = (hi + lo) * (2.0f / (float)N);
    // |c - c64| bound: the compensated sum, the cosines' representation, the
    // FP64 evaluation's own rounding (all far below 2^-40 sum |x| for N <= 128)
    // and the final roundings (covered by the |c| term)
    const float err = s1 * (2.0f / (float)N) * 0x1p-34f + 1e-30f;
    const float m = err + (k < d.B1 ? d.slack0 : d.slack1) + fabsf(c) * 0x1p-21f;
    bool decided;
    if (k < d.B1) {
      const uint32_t l0 = zone0_level32(c - m, d), l1 = zone0_level32(c + m, d);
      decided = l0 == l1;
      L = l0;
    } else {
      const double cd = ((double)hi + (double)lo) * (2.0 / (double)N);
      decided = zone1_decide(c, cd, (double)err * 2.0, m, d, L);
    }
    if (!decided) {
      const unsigned int slot = atomicAdd(p.fb_count, 1u);
      if (slot < p.fb_cap) {
        p.fb_list[slot] = g;
        return;  // k_enc_fallback writes the level
      }
      L = level_fp64(p, g);
    }
  }
  p.levels[g] = (uint8_t)L;
}

// The listed bins, one per thread, from their FP64 coefficients.
__global__ void __launch_bounds__(256) k_enc_fallback(EncParams p) {
  const unsigned int n = min(*p.fb_count, p.fb_cap);
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t g = p.fb_list[i];
    p.levels[g] = (uint8_t)level_fp64(p, g);
  }
}

// One thread per stream: Alg. 1's state over the code lengths, recorded at the
// start of every packing block; the words two blocks share are zeroed for the
// blocks' atomicOr; code and room checks; the stream's word count.
__global__ void __launch_bounds__(128) k_enc_scan(EncParams p) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.n_segs) return;
  const EncSeg sg = p.segs[s];
  const EncDomain d = p.doms[sg.domain];
  const uint8_t *lv = p.levels + sg.level_offset;
  const uint64_t L = sg.n_windows * d.E;
  const uint8_t *len = p.lens + d.code_off;
  PackState *const bs = p.blocks + sg.block_base;
  uint64_t w = 0;
  uint32_t bits = 0, count = 0;
  bool bad = false;
  // state update for symbol i of code length cl (> 0)
  auto step = [&](uint64_t i, uint32_t cl) {
    if ((i & (kPackBlock - 1)) == 0) {
      bs[i / kPackBlock] = PackState{w, bits, count};
      if (bits > 0 && w < sg.room) p.words[sg.word_offset + w] = 0;  // shared with the previous block
    }
    if (bits + cl > 64) {  // the codeword does not fit: the next word
      ++w;
      bits = 0;
      count = 0;
    }
    bits += cl;
    ++count;
  };
  // levels before the first 16-byte boundary one at a time
  uint64_t i = 0;
  const uint64_t to16 = (16u - (reinterpret_cast<uintptr_t>(lv) & 15u)) & 15u;
  const uint64_t head = to16 < L ? to16 : L;
  for (; i < head && !bad; ++i) {
    const uint32_t cl = __ldg(len + lv[i]);
    if (cl == 0)
      bad = true;
    else
      step(i, cl);
  }
  // then 16 at a time, the next chunk's load in flight while the current one is walked
  const uint64_t n16 = bad ? 0 : (L - i) / 16;
  uint4 nxt = n16 ? *reinterpret_cast<const uint4 *>(lv + i) : make_uint4(0u, 0u, 0u, 0u);
  for (uint64_t c = 0; c < n16 && !bad; ++c, i += 16) {
    const uint4 v = nxt;
    if (c + 1 < n16) nxt = *reinterpret_cast<const uint4 *>(lv + i + 16);
    const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
    uint32_t cl[16];
    bool zero = false;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      cl[j] = __ldg(len + ((vw[j >> 2] >> (8 * (j & 3))) & 0xffu));
      zero = zero || cl[j] == 0;
    }
    if (zero) {
      bad = true;
      break;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) step(i + j, cl[j]);
  }
  for (; i < L && !bad; ++i) {  // the tail
    const uint32_t cl = __ldg(len + lv[i]);
    if (cl == 0)
      bad = true;
    else
      step(i, cl);
  }
  if (bad) enc_flag(p.status, FPTC_ENC_FLAG_NO_CODE, s);
  const uint64_t total = w + (count > 0 ? 1u : 0u);
  if (!bad && total > sg.room) {
    enc_flag(p.status, FPTC_ENC_FLAG_ROOM, s);
    bad = true;
  }
  p.seg_bad[s] = bad ? 1u : 0u;
  p.n_words[s] = bad ? 0u : total;
}

// One thread per packing block: Alg. 1 from the block's recorded state.
__global__ void __launch_bounds__(128) k_enc_pack(EncParams p) {
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= p.n_blocks) return;
  const uint64_t s = last_leq(p.n_segs, b, [&](uint64_t i) { return p.segs[i].block_base; });
  if (p.seg_bad[s]) return;
  const EncSeg sg = p.segs[s];
  const EncDomain d = p.doms[sg.domain];
  const uint64_t j = b - sg.block_base;
  const uint64_t L = sg.n_windows * d.E;
  const uint64_t i0 = j * kPackBlock, i1 = i0 + kPackBlock < L ? i0 + kPackBlock : L;
  const uint8_t *lv = p.levels + sg.level_offset;
  const uint32_t *code = p.codes + d.code_off;
  const uint8_t *len = p.lens + d.code_off;
  unsigned long long *const out = reinterpret_cast<unsigned long long *>(p.words + sg.word_offset);
  uint8_t *const sl = p.symlen + sg.word_offset;
  const PackState st = p.blocks[b];
  uint64_t w = st.word;
  uint32_t bits = st.bits, count = st.count;
  const uint64_t first = w;
  const bool first_shared = bits > 0;  // part of the word came from the previous block
  uint64_t buffer = 0;
  auto put = [&](uint64_t word, uint64_t v) {
    if (word == first && first_shared)
      atomicOr(out + word, (unsigned long long)v);
    else
      out[word] = v;
  };
  auto step = [&](uint32_t sym) {
    const uint32_t cl = __ldg(len + sym);
    if (bits + cl > 64) {  // close the word
      put(w, buffer);
      sl[w] = (uint8_t)count;
      ++w;
      buffer = 0;
      bits = 0;
      count = 0;
    }
    buffer |= (uint64_t)__ldg(code + sym) << (64 - bits - cl);
    bits += cl;
    ++count;
  };
  for (uint64_t i = i0; i < i1;) {
    if ((reinterpret_cast<uintptr_t>(lv + i) & 15u) == 0 && i + 16 <= i1) {  // 16 levels in one load
      const uint4 v = *reinterpret_cast<const uint4 *>(lv + i);
      const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 16; ++j) step((vw[j >> 2] >> (8 * (j & 3))) & 0xffu);
      i += 16;
    } else {
      step(lv[i]);
      ++i;
    }
  }
  if (i1 == L) {  // the stream's last word
    if (count > 0) {
      put(w, buffer);
      sl[w] = (uint8_t)count;
    }
  } else {  // the open word continues in the next block (zeroed by the scan)
    atomicOr(out + w, (unsigned long long)buffer);
  }
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
  float *d_cosf = nullptr;
  PackState *d_blocks = nullptr;
  uint32_t *d_seg_bad = nullptr;
  unsigned long long *d_fb_list = nullptr;
  unsigned int *d_fb_count = nullptr;
  uint32_t fb_cap = 0;
  uint64_t n_blocks = 0;
  int sm_count = 1;
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
  cudaFree(e->d_cosf);
  cudaFree(e->d_blocks);
  cudaFree(e->d_seg_bad);
  cudaFree(e->d_fb_list);
  cudaFree(e->d_fb_count);
  cudaFree(e->d_codes);
  cudaFree(e->d_lens);
  cudaFree(e->d_status);
  cudaFree(e->d_lev_scratch);
}

struct EncDeleter {
  void operator()(fptc_encoder *e) const {
    enc_free(e);
    delete e;
  }
};

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
  p.cosf = e->d_cosf;
  p.blocks = e->d_blocks;
  p.seg_bad = e->d_seg_bad;
  p.fb_list = e->d_fb_list;
  p.fb_count = e->d_fb_count;
  p.fb_cap = e->fb_cap;
  p.n_blocks = e->n_blocks;
  p.codes = e->d_codes;
  p.lens = e->d_lens;
  p.status = e->d_status;
  p.n_segs = e->n_segs;
  p.n_levels = e->n_levels;
  return p;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

fptc_status fptc_encoder_create(fptc_encoder **enc, int device, const fptc_domain *domains, uint32_t n_domains,
                                const fptc_segment *segments, uint64_t n_segments) {
  return guarded([&]() -> fptc_status {
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
      x.A0f = (float)dm.scale[0];
      x.A1f = (float)dm.scale[1];
      x.muf = (float)dm.mu;
      x.d1f = (float)(dm.alpha1 * dm.scale[1]);
      x.d1 = dm.alpha1 * dm.scale[1];
      x.inv_A0f = dm.scale[0] > 1e-30 ? (float)(1.0 / dm.scale[0]) : 0.0f;
      x.inv_span1f = dm.scale[1] > 1e-30 && dm.scale[1] * (1.0 - dm.alpha1) > 0.0
                         ? (float)(1.0 / (dm.scale[1] - dm.alpha1 * dm.scale[1])) : 0.0f;
      x.inv_log1pmuf = (float)(1.0 / std::log1p(dm.mu));
      // 2^-18 of the zone scale: well above the FP32 evaluation error of either
      // map expressed in the coefficient (a few ulp of the scale: the maps'
      // arguments carry relative errors of a few 2^-24, over slopes of at most
      // mu / log1p(mu) and 1 / (1 - alpha1) per scale)
      x.slack0 = (float)(std::fabs(dm.scale[0]) * 0x1p-18);
      x.slack1 = (float)(std::fabs(dm.scale[1]) * 0x1p-18);
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
    // the same cosines as FP32 high and low parts, transposed per domain:
    // cosf[2 (cos_off + n E + k)] = hi, [+1] = lo, hi + lo = the FP64 cosine to 2^-48
    std::vector<float> cosf(2 * cosv.size());
    for (uint32_t d = 0; d < n_domains; ++d) {
      const EncDomain &x = doms[d];
      for (uint32_t k = 0; k < x.E; ++k)
        for (uint32_t n = 0; n < x.N; ++n) {
          const double c = cosv[x.cos_off + (size_t)k * x.N + n];
          const float h = (float)c;
          const size_t j = 2 * (x.cos_off + (size_t)n * x.E + k);
          cosf[j] = h;
          cosf[j + 1] = (float)(c - (double)h);
        }
    }
    std::vector<EncSeg> segs(n_segments);
    std::vector<uint64_t> level_off(n_segments);
    std::vector<std::pair<uint64_t, uint64_t>> rooms;
    uint64_t win = 0, lv = 0, blocks = 0;
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
      e.n_windows = (s.n_samples + dm.N - 1) / dm.N;
      e.block_base = blocks;
      e.domain = s.domain;
      e.pad = 0;
      level_off[i] = lv;
      win += e.n_windows;
      lv += e.n_windows * dm.E;
      blocks += (e.n_windows * dm.E + kPackBlock - 1) / kPackBlock;
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
    // the encoder under construction: released into *enc only on success, so
    // that an error return or an exception frees what it holds (destroyed
    // before g, with the encoder's device still current)
    std::unique_ptr<fptc_encoder, EncDeleter> owner(new fptc_encoder);
    fptc_encoder *const e = owner.get();
    e->device = device;
    e->n_segs = n_segments;
    e->n_windows = win;
    e->n_levels = lv;
    e->n_blocks = blocks;
    e->level_off = level_off;
    cudaError_t err = enc_upload(&e->d_segs, segs.data(), segs.size());
    if (err == cudaSuccess) err = enc_upload(&e->d_doms, doms.data(), doms.size());
    if (err == cudaSuccess) err = enc_upload(&e->d_cos, cosv.data(), cosv.size());
    if (err == cudaSuccess) err = enc_upload(&e->d_cosf, cosf.data(), cosf.size());
    if (err == cudaSuccess) err = cudaMalloc(&e->d_blocks, std::max<uint64_t>(blocks, 1) * sizeof(PackState));
    if (err == cudaSuccess) err = cudaMalloc(&e->d_seg_bad, std::max<uint64_t>(n_segments, 1) * sizeof(uint32_t));
    // room for the bins decided in FP64 (a few percent of them at most on signals; when it
    // fills, the level kernel decides the rest itself)
    e->fb_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(lv / 16, 4096), uint64_t(1) << 24);
    if (err == cudaSuccess) err = cudaMalloc(&e->d_fb_list, (size_t)e->fb_cap * sizeof(unsigned long long));
    if (err == cudaSuccess) err = cudaMalloc(&e->d_fb_count, sizeof(unsigned int));
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (err == cudaSuccess) err = enc_upload(&e->d_codes, codes.data(), codes.size());
    if (err == cudaSuccess) err = enc_upload(&e->d_lens, lens.data(), lens.size());
    if (err == cudaSuccess) {
      const EncStatus s0{0u, 0u, ~0ull};
      err = enc_upload(&e->d_status, &s0, 1);
    }
    if (err != cudaSuccess) return enc_cuda_fail(err, "encoder upload");
    *enc = owner.release();
    return FPTC_OK;
  });
}

void fptc_encoder_destroy(fptc_encoder *enc) {
  if (!enc) return;
  DevGuard g(enc->device);
  cudaDeviceSynchronize();
  EncDeleter()(enc);
}

uint64_t fptc_encoder_levels(const fptc_encoder *enc) { return enc ? enc->n_levels : 0; }

fptc_status fptc_encoder_level_offsets(const fptc_encoder *enc, uint64_t *offsets) {
  return guarded([&]() -> fptc_status {
    clear_error();
    if (!enc || (!offsets && enc->n_segs)) {
      set_error("NULL argument");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    std::copy(enc->level_off.begin(), enc->level_off.end(), offsets);
    return FPTC_OK;
  });
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
  if (!levels_given && enc->n_levels) {
    const uint64_t blocks = (enc->n_levels + 255) / 256;
    e = cudaMemsetAsync(enc->d_fb_count, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
      k_enc_levels<<<(unsigned)blocks, 256, 0, s>>>(p);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_enc_fallback<<<(unsigned)enc->sm_count * 8u, 256, 0, s>>>(p);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    k_enc_scan<<<(unsigned)((enc->n_segs + 127) / 128), 128, 0, s>>>(p);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && enc->n_blocks) {
    k_enc_pack<<<(unsigned)((enc->n_blocks + 127) / 128), 128, 0, s>>>(p);
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
