// The FPTC encoder on the GPU (include/fptc_encoder.h): Eq. 1, the three-zone
// quantizer of Sec. 3.2 and the SymLen packing of Alg. 1 for many streams.
//
//   k_enc_levels_w32  (every domain N = 32, E = 16) one thread per window: the
//                 window's 16 bins of Eq. 1 by the even/odd butterfly in FP32
//                 (dct32.cuh) with a bound on its error, and the zone
//                 quantizer bracketed by that bound.
//   k_enc_levels  (other shapes) one thread per (window, bin): the bin as a
//                 compensated FP32 dot product with a bound on its error.
//                 In both, every zone map is monotone in the coefficient, so
//                 when the levels at c - err and c + err agree the FP64
//                 coefficient (which lies between) has that level too;
//                 otherwise the bin goes to a list that k_enc_fallback
//                 computes again in FP64 (products and sums rounded
//                 separately, in sample order, then scaled by 2/N, as the host
//                 encoder does), one bin per lane, and quantizes from that.
//   k_enc_ref     one thread per packing block of kPackBlock symbols: Alg. 1
//                 on the block alone, entered with a word that starts at its
//                 first symbol (the reference packing): the words it closes
//                 and the state it ends in; then the next block of the stream
//                 packed from that state beside the next block's reference
//                 until the two start a word at the same symbol (from there
//                 on they coincide): the next block's transfer.
//   k_enc_scan    one warp per stream: the word counts added up block after
//                 block (a block entered in another state is walked again
//                 from the true one); each block's entry state; zeroes the
//                 words two blocks share; the stream's word count, room and
//                 code checks.
//   k_enc_pack    one thread per block: Alg. 1 from the block's entry state,
//                 whole words staged in shared memory and written out per
//                 warp, the words shared with the previous or next block with
//                 64-bit atomicOr (their codeword bits are disjoint), each
//                 word's symbol count by the block that closes it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <vector>

#include "dct32.cuh"
#include "device_util.cuh"
#include "fptc_codec.h"
#include "fptc_encoder.h"
#include "fptc_internal.h"
#include "host_util.h"

namespace fptc {
namespace {

constexpr uint32_t kPackBlock = 8192;  // symbols per packing block

struct EncDomain {
  uint32_t N, E, B1, B2;
  uint32_t cos_off;   // first entry of the E x N cosine tables (FP64 and FP32 copies)
  uint32_t code_off;  // first entry of the 256 codewords / lengths
  // FP32 forms for the fast evaluation of the quantizer
  float A0f, A1f, muf, d1f, inv_A0f, inv_span1f, inv_log1pmuf;
  float slack0, slack1;  // per zone: an input width that covers the FP32 evaluation error
  uint32_t on0, on1;     // A0 > 1e-30; A1 > 1e-30 and A1 > d1 (as the FP64 quantizer tests them): the zone is in use
  // zone 1 in units of the unscaled sum (c N / 2), for the window kernel's
  // branch-free first tier: d1, A1, slack1 scaled by N / 2 (exactly, N = 32),
  // and 126 / (A1 - d1), 127 / (A1 - d1) scaled by 2 / N
  float u1_d1, u1_A1, u1_slack, u1_kp, u1_kn;
  // zone 1's linear map may be evaluated in FP32 (A1 - d1 >= 2^-12 A1): the
  // FP32 roundings of A1 and d1 (2^-24 A1 each) then move the map's top by at
  // most 126 2^-23 / 2^-12 = 0.06 of a level; otherwise FP64 decides every
  // zone-1 bin outside the deadzone
  uint32_t z1_f32;
  uint32_t bnd_off;      // first of the domain's 2 x 255 boundaries of the host encoder's zone maps
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

struct RefEnd {
  uint32_t words;  // words the reference packing closes in the block (its last word stays open)
  uint32_t bits;   // bits used in that open word
  uint32_t count;  // its codewords
  uint32_t bad;    // a level of the block has no codeword
};

// What Alg. 1 does over one packing block entered in a given state.
struct BlockTrans {
  int32_t adj;     // met: the words it closes are the reference's plus adj; else the words it closes
  uint32_t bits;   // not met: the state it leaves the block in (bits of the open word
  uint32_t count;  // and its codewords); met: the reference's end state
  uint32_t flags;  // kTransMerged: it met the block's reference packing
};
constexpr uint32_t kTransMerged = 1u;

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
  RefEnd *ref_end;       // per packing block: the reference packing's end state
  BlockTrans *trans;     // per packing block: Alg. 1 over it from the state its predecessor's reference ends in
  const uint32_t *block_seg;  // per packing block: its segment
  const uint32_t *code_tab;   // per domain, 256 entries: codeword | length << 16
  const uint32_t *lv_seg;     // k_enc_levels_w32: the segment of each warp's first window
  const long long *bound_keys;  // per domain: zone 0's, then zone 1's 255 level boundaries (order keys)
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

// The host encoder's FP64 map of a zone (Eq. 2 or Eq. 3) is given as its 255
// ascending boundaries (the smallest double with level L or more, L = 1 ..
// 255, computed on the host from the host encoder's own map), stored as
// order keys: signed 64-bit integers that order like the doubles (the
// magnitude bits of a negative double flipped; a level no double reaches has
// the largest key), so that comparisons run on the integer pipe.  The level
// of a non-NaN c is the number of keys <= key(c).
__device__ __forceinline__ long long order_key(double c) {
  const long long b = __double_as_longlong(c);
  return b < 0 ? b ^ 0x7fffffffffffffffll : b;
}

__device__ __forceinline__ uint32_t level_by_keys(const long long *kb, long long kc) {
  uint32_t n = 0;
#pragma unroll
  for (uint32_t step = 128; step; step >>= 1)
    if (n + step <= 255u && __ldg(kb + n + step - 1) <= kc) n += step;
  return n;
}

__device__ __forceinline__ const long long *zone_keys(const EncParams &p, const EncDomain &d, uint32_t k) {
  return p.bound_keys + d.bnd_off + (k < d.B1 ? 0u : 255u);
}

// The host encoder's level of bin k for its FP64 coefficient c.
__device__ __forceinline__ uint32_t bin_level(const EncParams &p, uint32_t k, double c, const EncDomain &d) {
  if (k >= d.B2 || isnan(c)) return 128u;
  return level_by_keys(zone_keys(p, d, k), order_key(c));
}

// The level of bin k when the FP64 coefficient lies within err of cd: level
// L0 (an estimate) when both ends of [cd - err, cd + err] lie between
// boundaries L0 - 1 and L0 (two loads), else the map's level at both ends (the
// map is monotone); false when those differ or cd is not finite (the FP64
// coefficient decides).
__device__ __forceinline__ bool level_bracket64(const EncParams &p, uint32_t k, double cd, double err,
                                                uint32_t L0, const EncDomain &d, uint32_t &L) {
  if (k >= d.B2) {
    L = 128u;
    return true;
  }
  const double e = err + fabs(cd) * 0x1p-50;  // and the rounding of cd -+ e
  if (!(fabs(cd) + e <= 1.0e300)) return false;
  const long long *kb = zone_keys(p, d, k);
  const long long lo = order_key(cd - e), hi = order_key(cd + e);
  if ((L0 == 0u || __ldg(kb + L0 - 1) <= lo) && (L0 == 255u || hi < __ldg(kb + L0))) {
    L = L0;
    return true;
  }
  const uint32_t l0 = level_by_keys(kb, lo), l1 = level_by_keys(kb, hi);
  L = l0;
  return l0 == l1;
}

// Zone 0's map evaluated in FP32 (reciprocals, log1pf): off from the FP64
// evaluation by less than the zone's slack in the coefficient (both are close
// to the exact monotone map), so used only to bracket it.
__device__ __forceinline__ uint32_t zone0_level32(float c, const EncDomain &d) {
  if (!d.on0 || isnan(c)) return 128u;
  const float a = fminf(fabsf(c), d.A0f);
  const float q = log1pf(d.muf * (a * d.inv_A0f)) * d.inv_log1pmuf;
  const int v = c >= 0.0f ? 128 + (int)floorf(fmaf(127.0f, q, 0.5f)) : 128 - (int)floorf(fmaf(128.0f, q, 0.5f));
  return (uint32_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}

// A level near the FP32 coefficient c (the FP32 map at c; a start for
// level_bracket64, which checks it).
__device__ __forceinline__ uint32_t level_estimate(uint32_t k, float c, const EncDomain &d) {
  if (k >= d.B2) return 128u;
  if (k < d.B1) return zone0_level32(c, d);
  const float a = fabsf(c);
  if (!d.on1 || isnan(c) || a <= d.d1f) return 128u;
  const float r = fminf((fminf(a, d.A1f) - d.d1f) * d.inv_span1f, 1.0f);
  const int v = c > 0.0f ? 129 + (int)floorf(fmaf(r, 126.0f, 0.5f)) : 127 - (int)floorf(fmaf(r, 127.0f, 0.5f));
  return (uint32_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}

// Zone 1 decided in FP32 alone from c with |c - c64| <= m - slack1 (the first
// tier of the level kernels): the deadzone test against d1 rounded to FP32
// (|d1f - d1| <= 2^-24 A1, far inside the slack A1 2^-20 that m carries), then
// the linear map at both ends of the bracket.  Returns false when the bin has
// to be decided more closely.
__device__ __forceinline__ bool zone1_decide32(float c, float m, const EncDomain &d, uint32_t &L) {
  if (!d.on1 || isnan(c)) {
    L = 128u;
    return true;
  }
  const float a = fabsf(c);
  if (a + m < d.d1f) {
    L = 128u;
    return true;
  }
  if (a - m <= d.d1f || !d.z1_f32) return false;  // at the deadzone edge, or FP32 cannot map it
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

// Level of bin g (global level index) of segment s from the FP64 coefficient,
// computed as the host encoder does: products and sums rounded separately, in
// sample order, then scaled by 2/N.
__device__ __forceinline__ uint32_t level_fp64_seg(const EncParams &p, uint64_t g, uint64_t s) {
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
  return bin_level(p, k, __dmul_rn(a64, 2.0 / (double)d.N), d);
}

// FP64 list entries: level index (bits 0-39) and segment (bits 40-63).
__device__ __forceinline__ unsigned long long fb_entry(uint64_t g, uint64_t s) {
  return (unsigned long long)(g | (s << 40));
}
// A slot of the FP64 list for this thread, one atomic per warp (the lanes
// that call it at the same time share it); ~0u when the list is full.
__device__ __forceinline__ unsigned int fb_slot(const EncParams &p) {
  const uint32_t am = __activemask();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t leader = (uint32_t)(__ffs(am) - 1);
  unsigned int base = 0;
  if (lane == leader) base = atomicAdd(p.fb_count, (unsigned int)__popc(am));
  base = __shfl_sync(am, base, leader);
  const unsigned int slot = base + (unsigned int)__popc(am & ((1u << lane) - 1u));
  return slot < p.fb_cap ? slot : ~0u;
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
    // |c - c64| bound for c = hi + lo scaled in FP64: twice the compensated
    // sum's (2^-34 (2/N) sum |x|, which also covers the cosines' representation
    // and the FP64 evaluation's own rounding for N <= 128)
    const float err = s1 * (2.0f / (float)N) * 0x1p-34f + 1e-30f;
    const double cd = ((double)hi + (double)lo) * (2.0 / (double)N);
    const bool decided = level_bracket64(p, k, cd, 2.0 * (double)err, level_estimate(k, (float)cd, d), d, L);
    if (!decided) {
      const unsigned int slot = fb_slot(p);
      if (slot != ~0u) {
        p.fb_list[slot] = fb_entry(g, s);
        return;  // k_enc_fallback writes the level
      }
      L = level_fp64_seg(p, g, s);
    }
  }
  p.levels[g] = (uint8_t)L;
}

// First tier of k_enc_levels_w32 for the 16 bins of a window: levels into lv,
// the bins the bound cannot settle into the mask undecided (their level 0).
// T1: the zones of Table 1 (B1 = 2, B2 = 16), fixed per bin at compile time.
template <bool T1>
__device__ __forceinline__ void tier1_bins(const float (&a)[16], const float (&eb)[16], float err64,
                                           const EncDomain &d, uint32_t (&lv)[4], uint32_t &undecided) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float sc = k == 0 ? 4.0f / 32.0f : 2.0f / 32.0f;
    const float c = a[k] * sc;
    const bool z2 = T1 ? false : (uint32_t)k >= d.B2;
    const bool z0 = T1 ? k < 2 : (uint32_t)k < d.B1;
    uint32_t L = 128u;
    if (!z2) {
      const float err = eb[k] * sc + err64;
      const float m = err + (z0 ? d.slack0 : d.slack1) + fabsf(c) * 0x1p-21f;
      bool decided;
      if (z0) {
        const uint32_t l0 = zone0_level32(c - m, d), l1 = zone0_level32(c + m, d);
        decided = l0 == l1;
        L = l0;
      } else {
        decided = zone1_decide32(c, m, d, L);
      }
      if (!decided) {
        undecided |= 1u << k;
        L = 0u;
      }
    }
    lv[k >> 2] |= L << (8 * (k & 3));
  }
}

// The window kernel's first tier for Table 1's zones (B1 = 2, B2 = 16) when
// the window's samples are finite (so are its bins) and zone 1 is in use:
// bins 0 and 1 as in tier1_bins, bins 2 .. 15 branch-free in units of the
// unscaled sum a = c N / 2 (every constant scaled by the power of two N / 2
// = 16, so each comparison and rounding is the one zone1_decide32 makes on c,
// up to the level map's FP32 evaluation, whose error, a few ulp of a level
// index, is far inside the slack 2^-18 A1 that the bracket carries).
__device__ __forceinline__ void tier1_bins_fast(const float (&a)[16], const float (&eb)[16], float err64,
                                                const EncDomain &d, uint32_t (&lv)[4], uint32_t &undecided) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float sc = k == 0 ? 4.0f / 32.0f : 2.0f / 32.0f;
    const float c = a[k] * sc;
    const float m = eb[k] * sc + err64 + d.slack0 + fabsf(c) * 0x1p-21f;
    const uint32_t l0 = zone0_level32(c - m, d), l1 = zone0_level32(c + m, d);
    undecided |= l0 == l1 ? 0u : 1u << k;
    lv[0] |= (l0 == l1 ? l0 : 0u) << (8 * k);
  }
  const float base = err64 * 16.0f + d.u1_slack;  // err64 and slack1 in units of a
#pragma unroll
  for (int k = 2; k < 16; ++k) {
    const float ak = fabsf(a[k]);
    const float m = eb[k] + base + ak * 0x1p-21f;
    const float lo = ak - m, hi = ak + m;
    const bool dz = hi < d.u1_d1;              // settled: inside the deadzone
    const bool edge = lo <= d.u1_d1;           // else the deadzone edge is inside the bracket
    const bool pos = a[k] > 0.0f;
    const float kk = pos ? d.u1_kp : d.u1_kn;
    const int v0 = __float2int_rd(fmaf(fminf(lo, d.u1_A1) - d.u1_d1, kk, 0.5f));
    const int v1 = __float2int_rd(fmaf(fminf(hi, d.u1_A1) - d.u1_d1, kk, 0.5f));
    const bool und = !dz && (edge || v0 != v1);
    const uint32_t L = dz ? 128u : (und ? 0u : (uint32_t)(pos ? 129 + v0 : 127 - v0));
    undecided |= und ? 1u << k : 0u;
    lv[k >> 2] |= L << (8 * (k & 3));
  }
}

// Inclusive warp scan.
__device__ __forceinline__ uint32_t lane_prefix(uint32_t v, uint32_t lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (uint32_t)o) v += y;
  }
  return v;  // inclusive
}

constexpr uint32_t kLvThreads = 128;  // threads per CTA of k_enc_levels_w32 (4 warps)
constexpr uint32_t kTier2Inline = 8;  // a warp with more undecided bins settles them itself
constexpr uint32_t kLvGroups = 8;     // groups of 32 windows per warp, each loaded while the previous is computed
constexpr uint32_t kRowPitch = 36;    // floats per window row in shared memory (144 bytes: 16-byte reads conflict-free)

__device__ __forceinline__ uint32_t lds_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// 16 bytes, or src_bytes of them with zeros after (0: all zeros; src is not read)
__device__ __forceinline__ void cp_async_16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(lds_addr(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_4z(void *dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(lds_addr(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Where a window's samples are: its segment, the window within it, its first sample.
struct LvWin {
  uint64_t s = 0;           // segment
  uint64_t g0 = 0;          // its first level
  const float *src = nullptr;
  uint64_t avail = 0;       // samples from src on in the stream (>= 1), 0 for no window
};

__device__ __forceinline__ LvWin lv_window(const EncParams &p, uint64_t gw, uint64_t n_windows, uint64_t s_from) {
  LvWin r;
  r.s = s_from;
  if (gw >= n_windows) return r;
  r.g0 = gw * 16u;
  while (r.s + 1 < p.n_segs && p.segs[r.s + 1].level_offset <= r.g0) ++r.s;
  const EncSeg &sg = p.segs[r.s];
  const uint64_t i0 = ((r.g0 - sg.level_offset) >> 4) * 32u;
  r.avail = sg.n_samples - i0;
  r.src = p.x + sg.in_offset + i0;
  return r;
}

// The window's 32 samples into its shared-memory row, asynchronously (zero
// past the stream's end; no window: zeros).
__device__ __forceinline__ void lv_load_async(const EncParams &p, const LvWin &wn, float *row) {
  if (wn.avail >= 32 && (reinterpret_cast<uintptr_t>(wn.src) & 15u) == 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) cp_async_16(row + 4 * j, wn.src + 4 * j);
  } else {
    const float *base = wn.avail ? wn.src : p.x;  // a valid address where nothing is read
#pragma unroll 8
    for (int j = 0; j < 32; ++j)
      cp_async_4z(row + j, (uint64_t)j < wn.avail ? wn.src + j : base, (uint64_t)j < wn.avail ? 4u : 0u);
  }
}

// One thread per window, for encoders whose every domain has N = 32, E = 16:
// the window's 16 Eq. 1 bins at once by the even/odd butterfly in FP32, with
// a bound on each bin's error from the butterfly's own intermediate sums
// (dct32.cuh dct2_16_bounded; the exact scale 2/N, 4/N for bin 0), plus the
// FP64 encoder's own rounding; the zone quantizer is bracketed by that bound
// as in k_enc_levels.  Bins it cannot settle are computed again, spread over
// the warp's lanes, as compensated dot products; what those cannot settle goes
// to the FP64 list.  A warp takes kLvGroups groups of 32 consecutive windows;
// each group's samples come into shared memory by asynchronous copies while
// the warp computes the group before.
__global__ void __launch_bounds__(kLvThreads, 5) k_enc_levels_w32(EncParams p, uint64_t n_windows) {
  // per warp: two groups' samples (one row per window), and the second tier's
  // work list (window lane, bin), the windows' levels, segments, sample sums
  __shared__ __align__(16) float rows[kLvThreads / 32][2][32 * kRowPitch];
  __shared__ uint16_t work[kLvThreads / 32][512];
  __shared__ uint32_t lvs[kLvThreads / 32][32][4];
  __shared__ uint32_t segs_s[kLvThreads / 32][32];
  __shared__ float s1s[kLvThreads / 32][32];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const uint64_t chunk = (uint64_t)blockIdx.x * (kLvThreads / 32) + wid;
  if (chunk * kLvGroups * 32u >= n_windows) return;  // the whole warp
  const uint64_t first_group = chunk * kLvGroups;
  // the segment of the warp's first window from a table, then a step forward
  // per window (a warp's windows span few segments)
  const uint64_t s_first = p.lv_seg[chunk];
  LvWin cur = lv_window(p, first_group * 32u + lane, n_windows, s_first);
  lv_load_async(p, cur, rows[wid][0] + lane * kRowPitch);
  cp_async_commit_group();
#pragma unroll 1
  for (uint32_t t = 0; t < kLvGroups; ++t) {
    const uint64_t grp = first_group + t;
    if (grp * 32u >= n_windows) break;  // the whole warp
    // the next group's copies in flight
    LvWin nxt = cur;
    if (t + 1 < kLvGroups) {
      nxt = lv_window(p, (grp + 1) * 32u + lane, n_windows, cur.s);
      lv_load_async(p, nxt, rows[wid][(t + 1) & 1] + lane * kRowPitch);
    }
    cp_async_commit_group();
    cp_async_wait_group<1>();
    __syncwarp();
    const float *const xr = rows[wid][t & 1];
    const bool valid = cur.avail > 0;  // every lane stays for the warp's shuffles
    const uint64_t s = cur.s;
    const uint64_t g0 = cur.g0;
    const EncDomain d = p.doms[p.segs[s].domain];
    float x[32];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 v = *reinterpret_cast<const float4 *>(xr + lane * kRowPitch + 4 * j);
      x[4 * j] = v.x;
      x[4 * j + 1] = v.y;
      x[4 * j + 2] = v.z;
      x[4 * j + 3] = v.w;
    }
    float s1 = 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) s1 += fabsf(x[j]);
    float a[16], eb[16];
    dct32::dct2_16_bounded(x, a, eb);
    // |c - c64| <= the butterfly's bound for bin k (scaled like c) + the FP64 encoder's own rounding
    const float err64 = s1 * (2.0f / 32.0f) * 0x1p-40f + 1e-30f;
    uint32_t lv[4] = {0u, 0u, 0u, 0u};
    uint32_t undecided = 0;  // bins the butterfly's bound cannot settle
    if (d.B1 == 2u && d.B2 == 16u && d.z1_f32 && s1 <= 3.0e38f)  // Table 1's zones, finite bins
      tier1_bins_fast(a, eb, err64, d, lv, undecided);
    else if (d.B1 == 2u && d.B2 == 16u)  // the zone of every bin known at compile time
      tier1_bins<true>(a, eb, err64, d, lv, undecided);
    else
      tier1_bins<false>(a, eb, err64, d, lv, undecided);
    if (!valid) undecided = 0u;
    // second tier, spread over the warp's lanes: each undecided bin again as a
    // compensated FP32 dot product (|error| <= 2^-34 (2/N) sum |x|, as in
    // k_enc_levels); what that cannot settle goes to the FP64 list
    const uint32_t cnt = (uint32_t)__popc(undecided);
    const uint32_t incl = lane_prefix(cnt, lane);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total && total <= kTier2Inline) {  // a few: k_enc_fallback settles them (compensated, then FP64)
      uint64_t lo8 = ((uint64_t)lv[1] << 32) | lv[0], hi8 = ((uint64_t)lv[3] << 32) | lv[2];
      uint32_t u = undecided;
      while (u) {
        const uint32_t k = (uint32_t)(__ffs(u) - 1);
        u &= u - 1u;
        const unsigned int slot = fb_slot(p);
        if (slot != ~0u) {
          p.fb_list[slot] = fb_entry(g0 + k, s);  // its level (0 here) is written after the window's store
        } else {
          const uint64_t L = level_fp64_seg(p, g0 + k, s);
          if (k < 8)
            lo8 |= L << (8 * k);
          else
            hi8 |= L << (8 * (k - 8));
        }
      }
      lv[0] = (uint32_t)lo8;
      lv[1] = (uint32_t)(lo8 >> 32);
      lv[2] = (uint32_t)hi8;
      lv[3] = (uint32_t)(hi8 >> 32);
    } else if (total) {  // many (re-encoded signals): settled here, spread over the warp's lanes
      if (cnt) {
        segs_s[wid][lane] = (uint32_t)s;
        s1s[wid][lane] = s1;
        uint32_t u = undecided, o = incl - cnt;
        while (u) {
          work[wid][o++] = (uint16_t)((lane << 4) | (uint32_t)(__ffs(u) - 1));
          u &= u - 1u;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) lvs[wid][lane][q] = lv[q];
      __syncwarp();
      const uint64_t gw_base = grp * 32u;
      for (uint32_t i = lane; i < total; i += 32) {
        const uint32_t e = work[wid][i], own = e >> 4, k = e & 15u;
        const uint64_t so = segs_s[wid][own];
        const EncDomain od = p.doms[p.segs[so].domain];
        const float2 *ct = reinterpret_cast<const float2 *>(p.cosf) + od.cos_off + k;
        const float *xo = xr + own * kRowPitch;
        float hi = 0.0f, lo = 0.0f;
#pragma unroll 8
        for (int n = 0; n < 32; ++n) {
          const float xv = xo[n];
          const float2 cs = ct[(size_t)n * 16u];
          const float pr = __fmul_rn(xv, cs.x);
          const float pe = __fadd_rn(__fmaf_rn(xv, cs.x, -pr), __fmul_rn(xv, cs.y));
          const float tt = __fadd_rn(hi, pr);
          const float bp = __fsub_rn(tt, hi);
          lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(tt, bp)), __fsub_rn(pr, bp)), pe));
          hi = tt;
        }
        const float err2 = s1s[wid][own] * (2.0f / 32.0f) * 0x1p-34f + 1e-30f;
        const double cd = ((double)hi + (double)lo) * (2.0 / 32.0);
        uint32_t L = 0u;
        const bool decided =
            level_bracket64(p, k, cd, 2.0 * (double)err2, level_estimate(k, (float)cd, od), od, L);
        const uint64_t g = (gw_base + own) * 16u + k;
        if (!decided) {
          const unsigned int slot = fb_slot(p);
          if (slot != ~0u) {
            p.fb_list[slot] = fb_entry(g, so);
            L = 0u;  // k_enc_fallback writes this level after the window's store
          } else {
            L = level_fp64_seg(p, g, so);
          }
        }
        reinterpret_cast<uint8_t *>(lvs[wid][own])[k] = (uint8_t)L;
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 4; ++q) lv[q] = lvs[wid][lane][q];
    }
    if (valid) {
      uint8_t *const dst = p.levels + g0;
      if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        *reinterpret_cast<uint4 *>(dst) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) dst[k] = (uint8_t)(lv[k >> 2] >> (8 * (k & 3)));
      }
    }
    __syncwarp();  // every lane is done with this group's rows and tier-2 lists before they are refilled
    cur = nxt;
  }
  cp_async_wait_group<0>();
}

// ---- SymLen packing (Alg. 1) in parallel over blocks of kPackBlock symbols ----
// Alg. 1 closes a word when the next codeword does not fit, so where words
// start inside a block depends only on the state the block is entered with
// (the bits already used in the open word).  Greedy packings entered with
// different states soon start a word at the same symbol, and from there on
// they coincide.  Call the packing of a block entered with a word that starts
// at its first symbol the block's reference packing.  A block whose packing
// meets its reference ends in the reference's end state, whatever state it
// was entered with; so in the usual case every block but a stream's first is
// entered in the state its predecessor's reference ends in.  k_enc_ref packs
// block b as its reference does (the words it closes, the state it ends in),
// then walks block b + 1 from that end state beside block b + 1's reference
// until the two start a word at the same symbol: the transfer of block b + 1,
// from the state it is entered in when block b met its reference.  k_enc_scan
// adds the word counts up along each stream; a block whose predecessor never
// met its reference (constant code lengths can do that) was entered in
// another state, and the scan walks it again from the true one.

// 16 levels from lv + i (zero past n) as one 16-byte vector.
__device__ __forceinline__ uint4 load_raw16(const uint8_t *lv, uint64_t i, uint64_t n) {
  if (i + 16 <= n && (reinterpret_cast<uintptr_t>(lv + i) & 15u) == 0) return *reinterpret_cast<const uint4 *>(lv + i);
  uint32_t t[4] = {0u, 0u, 0u, 0u};
  for (uint32_t r = 0; r < 16 && i + r < n; ++r) t[r >> 2] |= (uint32_t)lv[i + r] << (8 * (r & 3));
  return make_uint4(t[0], t[1], t[2], t[3]);
}

// 64 levels from lv + i (zero past n) as four 16-byte vectors.
__device__ __forceinline__ void load_raw64(const uint8_t *lv, uint64_t i, uint64_t n, uint4 (&v)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = load_raw16(lv, i + 16 * q, n);
}

// Alg. 1 over 64 levels of the reference packing (FULL: all 64 exist).
template <bool FULL>
__device__ __forceinline__ void ref_step64(const uint4 (&v)[4], uint32_t i, uint32_t nb, const uint8_t *len,
                                           uint32_t &words, uint32_t &bits, uint32_t &count, bool &bad) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t vw[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
    uint32_t cl[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) cl[j] = __ldg(len + ((vw[j >> 2] >> (8 * (j & 3))) & 0xffu));
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (!FULL && i + 16 * q + j >= nb) break;
      const uint32_t c = cl[j];
      bad = bad || c == 0u;
      const bool start = count == 0u || bits + c > 64u;  // a word starts here
      words += (start && count) ? 1u : 0u;
      bits = (start ? 0u : bits) + c;
      count = (start ? 0u : count) + 1u;
    }
  }
}

// One thread per packing block b: its reference packing, then the transfer
// of block b + 1 (when it is in the same stream) entered in the state the
// reference of b ends in.
__global__ void __launch_bounds__(128) k_enc_ref(EncParams p) {
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= p.n_blocks) return;
  const EncSeg sg = p.segs[p.block_seg[b]];
  const EncDomain d = p.doms[sg.domain];
  const uint64_t L = sg.n_windows * d.E;
  const uint64_t i0 = (b - sg.block_base) * kPackBlock;
  const uint32_t nb = (uint32_t)(L - i0 < kPackBlock ? L - i0 : kPackBlock);
  const uint8_t *lv = p.levels + sg.level_offset + i0;
  const uint8_t *len = p.lens + d.code_off;
  uint32_t words = 0, bits = 0, count = 0;
  bool bad = false;
  // block b + 1 of the same stream, if any
  const uint32_t nb2 = i0 + nb < L ? (uint32_t)(L - i0 - nb < kPackBlock ? L - i0 - nb : kPackBlock) : 0u;
  // 64 levels per step, the next 64 in flight
  uint4 v[4], vn[4];
  load_raw64(lv, 0, nb, v);
  for (uint32_t i = 0; i < nb; i += 64) {
    if (i + 64 < nb) load_raw64(lv, i + 64, nb, vn);
    if (i + 64 <= nb)
      ref_step64<true>(v, i, nb, len, words, bits, count, bad);
    else
      ref_step64<false>(v, i, nb, len, words, bits, count, bad);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = vn[q];
  }
  p.ref_end[b] = RefEnd{words, bits, count, bad ? 1u : 0u};
  if (b == sg.block_base) p.trans[b] = BlockTrans{0, 0u, 0u, kTransMerged};  // a stream's first block packs as its reference
  if (nb2 == 0) return;
  // block b + 1: Alg. 1 from (bits, count) and from a fresh word side by side
  const uint8_t *lv2 = lv + nb;
  uint32_t rb = 0, rc = 0, closes = 0, r = 0;
  bool met = false;
  for (uint32_t i = 0; i < nb2 && !met; i += 16) {
    const uint4 u = load_raw16(lv2, i, nb2);
    const uint32_t vw[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (i + j >= nb2) break;
      const uint32_t c = __ldg(len + ((vw[j >> 2] >> (8 * (j & 3))) & 0xffu));
      const bool rs = rc == 0u || rb + c > 64u;  // the reference starts a word here
      const bool ts = bits + c > 64u;            // so does the packing from (bits, count)
      if (rs && ts) {
        met = true;
        break;
      }
      r += rs ? 1u : 0u;
      closes += ts ? 1u : 0u;
      rb = (rs ? 0u : rb) + c;
      rc = (rs ? 0u : rc) + 1u;
      bits = (ts ? 0u : bits) + c;
      count = (ts ? 0u : count) + 1u;
    }
  }
  // met: the word open before the meeting symbol closes there, then come the
  // reference's words but the r that start before it
  p.trans[b + 1] = met ? BlockTrans{(int32_t)(closes + 1u) - (int32_t)r, 0u, 0u, kTransMerged}
                       : BlockTrans{(int32_t)closes, bits, count, 0u};
}

// Word starts of Alg. 1 among symbols from .. valid - 1 of a chunk of 32
// (S: inclusive prefix of the chunk's code lengths, per lane), entered in
// (bits, count); a word that starts at the chunk's first symbol because none
// is open (count == 0) is one too.  One ballot per word start; the state is
// carried over.
__device__ __forceinline__ uint32_t chunk_starts(uint32_t S, uint32_t lane, uint32_t valid, uint32_t &bits,
                                                 uint32_t &count) {
  uint32_t mask = count == 0u ? 1u : 0u;
  uint32_t from = 0;
  while (true) {
    const uint32_t pre = from ? __shfl_sync(0xffffffffu, S, from - 1) : 0u;
    const uint32_t over = __ballot_sync(0xffffffffu, lane >= from && lane < valid && bits + (S - pre) > 64u);
    if (over == 0) {  // the rest of the chunk fits the open word
      bits += __shfl_sync(0xffffffffu, S, valid - 1) - pre;
      count += valid - from;
      return mask;
    }
    from = (uint32_t)(__ffs(over) - 1);  // a word starts at symbol from
    mask |= 1u << from;
    bits = 0;
    count = 0;
  }
}

// The transfer of block b entered in (bits, count > 0), by the whole warp:
// Alg. 1 from that state and the block's reference side by side, 32 symbols
// at a time (a warp scan of their code lengths; each word start one ballot),
// until both start a word at the same symbol.  Levels arrive 128 per round
// trip (a 4-byte load per lane), the next 128 in flight.
__device__ BlockTrans walk_block(const EncParams &p, const EncSeg &sg, const EncDomain &d, uint64_t b, uint32_t bits,
                                 uint32_t count, uint32_t lane) {
  const uint64_t L = sg.n_windows * d.E;
  const uint64_t i0 = (b - sg.block_base) * kPackBlock;
  const uint32_t nb = (uint32_t)(L - i0 < kPackBlock ? L - i0 : kPackBlock);
  const uint8_t *lv = p.levels + sg.level_offset + i0;
  const uint8_t *len = p.lens + d.code_off;
  uint32_t rb = 0, rc = 0, closes = 0, r = 0;
  auto fetch = [&](uint32_t at) -> uint32_t {  // levels at .. at + 127, four per lane
    const uint32_t o = at + 4 * lane;
    if (o + 4 <= nb && (reinterpret_cast<uintptr_t>(lv + o) & 3u) == 0) return *reinterpret_cast<const uint32_t *>(lv + o);
    uint32_t t = 0;
    for (uint32_t q = 0; q < 4 && o + q < nb; ++q) t |= (uint32_t)lv[o + q] << (8 * q);
    return t;
  };
  uint32_t cur = fetch(0);
  for (uint32_t at = 0; at < nb; at += 128) {
    const uint32_t nxt = at + 128 < nb ? fetch(at + 128) : 0u;
#pragma unroll 1
    for (uint32_t k = 0; k < 4; ++k) {
      const uint32_t c = at + 32 * k;
      if (c >= nb) break;
      const uint32_t valid = nb - c < 32 ? nb - c : 32;
      const uint32_t vw = __shfl_sync(0xffffffffu, cur, 8 * k + (lane >> 2));
      const uint32_t cl = lane < valid ? __ldg(len + ((vw >> (8 * (lane & 3))) & 0xffu)) : 0u;
      const uint32_t S = lane_prefix(cl, lane);
      const uint32_t rm = chunk_starts(S, lane, valid, rb, rc);
      const uint32_t tm = chunk_starts(S, lane, valid, bits, count);
      const uint32_t both = rm & tm;
      if (both) {  // they meet at symbol c + t
        const uint32_t before = (1u << (__ffs(both) - 1)) - 1u;
        closes += __popc(tm & before);
        r += __popc(rm & before);
        return BlockTrans{(int32_t)(closes + 1u) - (int32_t)r, 0u, 0u, kTransMerged};
      }
      closes += __popc(tm);
      r += __popc(rm);
    }
    cur = nxt;
  }
  return BlockTrans{(int32_t)closes, bits, count, 0u};
}

// One warp per stream: the true packing state block after block from the
// blocks' transfers, 32 blocks at a time (a warp scan of their word counts);
// each block's entry state for k_enc_pack; the words two blocks share are
// zeroed for the blocks' atomicOr; code and room checks; the stream's word
// count.  A block entered in another state than its transfer assumed (its
// predecessor never met its reference) is walked again from the true state.
__global__ void __launch_bounds__(128) k_enc_scan(EncParams p) {
  const uint64_t s = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  if (s >= p.n_segs) return;  // the whole warp
  const EncSeg sg = p.segs[s];
  const EncDomain d = p.doms[sg.domain];
  const uint64_t L = sg.n_windows * d.E;
  const uint64_t nblk = (L + kPackBlock - 1) / kPackBlock;
  uint64_t w = 0;  // the open word (words closed so far)
  uint32_t bits = 0, count = 0;
  bool assumed = true;  // the next block is entered in the state its transfer assumed
  bool bad = false;
  uint64_t jb = 0;
  while (jb < nblk) {
    const uint64_t b0 = sg.block_base + jb;
    if (!assumed) {
      if (lane == 0) {
        p.blocks[b0] = PackState{w, bits, count};
        if (bits > 0 && w < sg.room) p.words[sg.word_offset + w] = 0;  // shared with the previous block
      }
      const RefEnd re = p.ref_end[b0];
      if (re.bad) {
        bad = true;
        break;
      }
      const BlockTrans t = walk_block(p, sg, d, b0, bits, count, lane);
      const bool met = (t.flags & kTransMerged) != 0;
      w += (uint64_t)((int64_t)t.adj + (met ? (int64_t)re.words : 0));
      bits = met ? re.bits : t.bits;
      count = met ? re.count : t.count;
      assumed = met;
      ++jb;
      continue;
    }
    const uint32_t n = nblk - jb < 32 ? (uint32_t)(nblk - jb) : 32u;
    BlockTrans t{0, 0u, 0u, 0u};
    RefEnd re{0u, 0u, 0u, 0u};
    if (lane < n) {
      t = p.trans[b0 + lane];
      re = p.ref_end[b0 + lane];
    }
    const bool met = (t.flags & kTransMerged) != 0;
    const uint32_t delta = (uint32_t)(t.adj + (met ? (int32_t)re.words : 0));
    const uint32_t xb = met ? re.bits : t.bits, xc = met ? re.count : t.count;  // the state it leaves
    const uint32_t badm = __ballot_sync(0xffffffffu, lane < n && re.bad);
    const uint32_t open = __ballot_sync(0xffffffffu, lane < n && !met);
    // the blocks entered as assumed: up to the first that did not meet its
    // reference (it is itself one), before the first bad one
    uint32_t m = n;
    if (open) m = min(m, (uint32_t)__ffs(open));
    const uint32_t first_bad = badm ? (uint32_t)(__ffs(badm) - 1) : 32u;
    m = min(m, first_bad);
    uint32_t eb = __shfl_up_sync(0xffffffffu, xb, 1), ec = __shfl_up_sync(0xffffffffu, xc, 1);
    if (lane == 0) {
      eb = bits;
      ec = count;
    }
    const uint32_t dl = lane < m ? delta : 0u;
    const uint32_t incl = lane_prefix(dl, lane);
    const uint64_t we = w + (incl - dl);
    if (lane < m) {
      p.blocks[b0 + lane] = PackState{we, eb, ec};
      if (eb > 0 && we < sg.room) p.words[sg.word_offset + we] = 0;  // shared with the previous block
    }
    if (m > 0) {
      w += __shfl_sync(0xffffffffu, incl, m - 1);
      bits = __shfl_sync(0xffffffffu, xb, m - 1);
      count = __shfl_sync(0xffffffffu, xc, m - 1);
      assumed = ((open >> (m - 1)) & 1u) == 0u;
    }
    jb += m;
    if (badm && m == first_bad) {
      bad = true;
      break;
    }
  }
  if (lane == 0) {
    if (bad) enc_flag(p.status, FPTC_ENC_FLAG_NO_CODE, s);
    const uint64_t total = w + (count > 0 ? 1u : 0u);
    if (!bad && total > sg.room) {
      enc_flag(p.status, FPTC_ENC_FLAG_ROOM, s);
      bad = true;
    }
    p.seg_bad[s] = bad ? 1u : 0u;
    p.n_words[s] = bad ? 0u : total;
  }
}

// Level of listed bin g of segment s from its compensated FP32 coefficient (as
// in k_enc_levels: |error| <= 2^-34 (2/N) sum |x|); false when that bound
// cannot settle it.
__device__ __forceinline__ bool level_compensated(const EncParams &p, uint64_t g, uint64_t s, uint32_t &L) {
  const EncSeg sg = p.segs[s];
  const EncDomain d = p.doms[sg.domain];
  const uint64_t local = g - sg.level_offset;
  const uint64_t w = local / d.E;
  const uint32_t k = (uint32_t)(local - w * d.E);
  const uint64_t avail = sg.n_samples - w * d.N;
  const uint32_t nn = avail < d.N ? (uint32_t)avail : d.N;
  const float *src = p.x + sg.in_offset + w * d.N;
  const float2 *ct = reinterpret_cast<const float2 *>(p.cosf) + d.cos_off + k;
  float hi = 0.0f, lo = 0.0f, s1 = 0.0f;
  auto step = [&](float xv, float2 cs) {
    const float pr = __fmul_rn(xv, cs.x);
    const float pe = __fadd_rn(__fmaf_rn(xv, cs.x, -pr), __fmul_rn(xv, cs.y));
    const float t = __fadd_rn(hi, pr);
    const float bp = __fsub_rn(t, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(pr, bp)), pe));
    hi = t;
    s1 += fabsf(xv);
  };
  if (d.N == 32 && nn == 32 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    // a whole window: its samples and cosines requested at once, the same
    // operations in the same order as below
    float xv[32];
    float2 cs[32];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + j);
      xv[4 * j] = v.x;
      xv[4 * j + 1] = v.y;
      xv[4 * j + 2] = v.z;
      xv[4 * j + 3] = v.w;
    }
#pragma unroll
    for (int n = 0; n < 32; ++n) cs[n] = __ldg(ct + (size_t)n * d.E);
#pragma unroll
    for (int n = 0; n < 32; ++n) step(xv[n], cs[n]);
  } else {
    for (uint32_t n = 0; n < nn; ++n) step(__ldg(src + n), __ldg(ct + (size_t)n * d.E));
  }
  const float err2 = s1 * (2.0f / (float)d.N) * 0x1p-34f + 1e-30f;
  const double cd = ((double)hi + (double)lo) * (2.0 / (double)d.N);
  return level_bracket64(p, k, cd, 2.0 * (double)err2, level_estimate(k, (float)cd, d), d, L);
}

// The listed bins, one per thread: from their compensated FP32 coefficient
// where its bound settles the level, else from their FP64 coefficient.
__global__ void __launch_bounds__(256) k_enc_fallback(EncParams p) {
  const unsigned int n = min(*p.fb_count, p.fb_cap);
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long e = p.fb_list[i];
    const uint64_t g = e & ((1ull << 40) - 1ull), s = e >> 40;
    uint32_t L;
    if (!level_compensated(p, g, s, L)) L = level_fp64_seg(p, g, s);
    p.levels[g] = (uint8_t)L;
  }
}

// k_enc_pack: one thread per packing block, Alg. 1 from the block's entry
// state, branch-free per codeword (one table load gives code and length).  A
// word that closes is staged in shared memory; after every 64 codewords the
// warp writes its lanes' staged words out together, two lanes' words per
// round (16 lanes each), so that a store instruction writes one lane's
// consecutive words instead of one word of each of 32 streams.  The first
// word of a block entered with bits already used is shared with the previous
// block and goes out with a 64-bit atomicOr (the two parts' bits are
// disjoint; the scan zeroed it), as does the word a block leaves open for the
// next.  Each word's symbol count is written by the block that closes it.
constexpr uint32_t kStageWords = 16;  // words that can close in 64 codewords (>= 4 codewords each: lmax <= 16)
constexpr uint32_t kStagePitch = 17;  // per lane, padded against bank conflicts
constexpr uint32_t kPackWarps = 4;

struct PackLane {
  const uint8_t *lv = nullptr;    // the block's levels
  const uint32_t *tab = nullptr;  // code | length << 16 per level
  uint64_t g0 = 0;                // index in p.words of the block's first word
  uint32_t n = 0;                 // codewords of the block (0: no work)
  uint32_t bits = 0, count = 0;   // Alg. 1's state
  uint32_t wf = 0, ns = 0;        // words of the block written out; staged
  uint64_t buffer = 0;            // the open word's codewords, left-aligned
  bool shared_first = false;      // the block's first word holds bits of the previous block
};

template <bool FULL>
__device__ __forceinline__ void pack_step64(PackLane &t, const uint4 (&v)[4], uint32_t i, unsigned long long *sw,
                                            uint8_t *sc) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t vw[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (!FULL && i + 16 * q + j >= t.n) break;
      const uint32_t e = __ldg(t.tab + ((vw[j >> 2] >> (8 * (j & 3))) & 0xffu));
      const uint32_t cl = e >> 16;
      const bool close = t.bits + cl > 64u;
      if (close) {
        sw[t.ns] = t.buffer;
        sc[t.ns] = (uint8_t)t.count;
      }
      t.ns += close ? 1u : 0u;
      t.bits = (close ? 0u : t.bits) + cl;
      t.count = (close ? 0u : t.count) + 1u;
      t.buffer = (close ? 0ull : t.buffer) | ((uint64_t)(e & 0xffffu) << (64u - t.bits));
    }
  }
}

__global__ void __launch_bounds__(kPackWarps * 32) k_enc_pack(EncParams p) {
  __shared__ unsigned long long stage_w[kPackWarps][32 * kStagePitch];
  __shared__ uint8_t stage_c[kPackWarps][32 * kStageWords];
  __shared__ uint4 stage_i[kPackWarps][32];  // per lane: first staged word (index in p.words), count, shared flag
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  unsigned long long *const sw = stage_w[wid] + lane * kStagePitch;
  uint8_t *const sc = stage_c[wid] + lane * kStageWords;
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  PackLane t;
  bool last = false;  // the block ends its stream
  if (b < p.n_blocks) {
    const uint32_t s = p.block_seg[b];
    if (!p.seg_bad[s]) {
      const EncSeg sg = p.segs[s];
      const EncDomain d = p.doms[sg.domain];
      const uint64_t L = sg.n_windows * d.E;
      const uint64_t i0 = (b - sg.block_base) * kPackBlock;
      t.n = (uint32_t)(L - i0 < kPackBlock ? L - i0 : kPackBlock);
      t.lv = p.levels + sg.level_offset + i0;
      t.tab = p.code_tab + d.code_off;
      const PackState st = p.blocks[b];
      t.g0 = sg.word_offset + st.word;
      t.bits = st.bits;
      t.count = st.count;
      t.shared_first = st.bits > 0;
      last = i0 + t.n == L;
    }
  }
  const uint32_t nmax = __reduce_max_sync(0xffffffffu, t.n);
  uint4 v[4], vn[4];
  if (t.n) load_raw64(t.lv, 0, t.n, v);
  for (uint32_t i = 0; i < nmax; i += 64) {
    if (i < t.n) {
      if (i + 64 < t.n) load_raw64(t.lv, i + 64, t.n, vn);
      if (i + 64 <= t.n)
        pack_step64<true>(t, v, i, sw, sc);
      else
        pack_step64<false>(t, v, i, sw, sc);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = vn[q];
    }
    // the warp writes its staged words: round r, half h writes lane 2 r + h's
    stage_i[wid][lane] = make_uint4((uint32_t)(t.g0 + t.wf), (uint32_t)((t.g0 + t.wf) >> 32), t.ns,
                                    t.shared_first && t.wf == 0u ? 1u : 0u);
    __syncwarp();
    const uint32_t h = lane >> 4, j = lane & 15u;
#pragma unroll 4
    for (uint32_t r = 0; r < 16; ++r) {
      const uint32_t src = 2u * r + h;
      const uint4 si = stage_i[wid][src];
      if (j < si.z) {
        const uint64_t g = ((uint64_t)si.y << 32 | si.x) + j;
        const unsigned long long wv = stage_w[wid][src * kStagePitch + j];
        if (j == 0 && si.w)
          atomicOr(reinterpret_cast<unsigned long long *>(p.words) + g, wv);
        else
          p.words[g] = wv;
        p.symlen[g] = stage_c[wid][src * kStageWords + j];
      }
    }
    __syncwarp();
    t.wf += t.ns;
    t.ns = 0;
  }
  if (t.n) {
    unsigned long long *const wp = reinterpret_cast<unsigned long long *>(p.words) + t.g0 + t.wf;
    if (last) {  // the stream's last word
      if (t.count > 0) {
        if (t.wf == 0 && t.shared_first)
          atomicOr(wp, (unsigned long long)t.buffer);
        else
          *wp = t.buffer;
        p.symlen[t.g0 + t.wf] = (uint8_t)t.count;
      }
    } else {  // the open word continues in the next block (zeroed by the scan)
      atomicOr(wp, (unsigned long long)t.buffer);
    }
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
  RefEnd *d_ref_end = nullptr;              // [n_blocks]
  BlockTrans *d_trans = nullptr;            // [n_blocks]
  uint32_t *d_block_seg = nullptr;          // [n_blocks]
  uint32_t *d_code_tab = nullptr;           // [n_domains][256]
  uint32_t *d_lv_seg = nullptr;             // [warps of k_enc_levels_w32]
  long long *d_bound_keys = nullptr;        // [n_domains][2][255]
  bool w32 = false;               // every domain N = 32, E = 16: the window-per-thread level kernel
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
  cudaFree(e->d_ref_end);
  cudaFree(e->d_trans);
  cudaFree(e->d_block_seg);
  cudaFree(e->d_code_tab);
  cudaFree(e->d_lv_seg);
  cudaFree(e->d_bound_keys);
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
  p.ref_end = e->d_ref_end;
  p.trans = e->d_trans;
  p.block_seg = e->d_block_seg;
  p.code_tab = e->d_code_tab;
  p.lv_seg = e->d_lv_seg;
  p.bound_keys = e->d_bound_keys;
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
    std::vector<uint32_t> code_tab;
    std::vector<double> bounds(2 * 255 * (size_t)n_domains);
    std::vector<long long> bound_keys(bounds.size());
    for (uint32_t d = 0; d < n_domains; ++d) {
      const fptc_domain &dm = domains[d];
      fptc_status st = fptc_validate_domain(&dm);
      if (st != FPTC_OK) return st;
      EncDomain &x = doms[d];
      x.N = dm.N;
      x.E = dm.E;
      x.B1 = dm.B1;
      x.B2 = dm.B2;
      x.A0f = (float)dm.scale[0];
      x.A1f = (float)dm.scale[1];
      x.muf = (float)dm.mu;
      const double d1 = dm.alpha1 * dm.scale[1];  // as the FP64 quantizer computes it
      x.d1f = (float)d1;
      x.inv_A0f = dm.scale[0] > 1e-30 ? (float)(1.0 / dm.scale[0]) : 0.0f;
      x.inv_span1f = dm.scale[1] > 1e-30 && dm.scale[1] * (1.0 - dm.alpha1) > 0.0
                         ? (float)(1.0 / (dm.scale[1] - dm.alpha1 * dm.scale[1])) : 0.0f;
      x.inv_log1pmuf = (float)(1.0 / std::log1p(dm.mu));
      // 2^-18 of the zone scale: well above the FP32 evaluation error of either
      // map expressed in the coefficient (a few ulp of the scale: the maps'
      // arguments carry relative errors of a few 2^-24, over slopes of at most
      // mu / log1p(mu) and 1 / (1 - alpha1) per scale)
      x.slack0 = (float)(std::fabs(dm.scale[0]) * 0x1p-18);
      // zone 1's map is linear: its FP32 evaluation errs by a few 2^-24 A1 in
      // the coefficient (an emulation of both FP32 forms still brackets the
      // FP64 map with 2^-22 A1)
      x.slack1 = (float)(std::fabs(dm.scale[1]) * 0x1p-20);
      x.on0 = dm.scale[0] > 1e-30 ? 1u : 0u;
      // zone 1 is in use when A1 > 1e-30 and its linear part is not empty: with
      // alpha1 = 1 every |c| <= min(|c|, A1) <= d1, all level 128
      x.on1 = dm.scale[1] > 1e-30 && dm.scale[1] - d1 > 0.0 ? 1u : 0u;
      {
        const double h = dm.N / 2.0, span = dm.scale[1] - d1;
        x.u1_d1 = (float)(d1 * h);
        x.u1_A1 = (float)(dm.scale[1] * h);
        x.u1_slack = (float)(std::fabs(dm.scale[1]) * 0x1p-20 * h);
        x.u1_kp = span > 0.0 ? (float)(126.0 / span / h) : 0.0f;
        x.u1_kn = span > 0.0 ? (float)(127.0 / span / h) : 0.0f;
        x.z1_f32 = x.on1 && span >= dm.scale[1] * 0x1p-12 ? 1u : 0u;
      }
      // the host encoder's zone maps as boundaries: the levels of the second
      // and third tiers are those maps' own
      x.bnd_off = 2 * 255 * d;
      host_zone_bounds(dm, 0, bounds.data() + x.bnd_off);
      host_zone_bounds(dm, 1, bounds.data() + x.bnd_off + 255);
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
        code_tab.push_back(c[s] | (uint32_t)dm.code_len[s] << 16);  // codes have <= lmax <= 16 bits
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
    std::vector<uint32_t> block_seg;
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
      const uint64_t nb = (e.n_windows * dm.E + kPackBlock - 1) / kPackBlock;
      blocks += nb;
      block_seg.insert(block_seg.end(), nb, (uint32_t)i);
      if (s.n_words) rooms.push_back({s.word_offset, s.word_offset + s.n_words});
    }
    std::sort(rooms.begin(), rooms.end());
    for (size_t i = 1; i < rooms.size(); ++i)
      if (rooms[i].first < rooms[i - 1].second) {
        set_error("segment rooms overlap at word %llu", (unsigned long long)rooms[i].first);
        return FPTC_ERR_INVALID_ARGUMENT;
      }
    if (lv >= (uint64_t(1) << 40) || n_segments >= (uint64_t(1) << 24)) {  // the FP64 list packs both in 64 bits
      set_error("an encoder takes at most 2^40 levels and 2^24 segments");
      return FPTC_ERR_UNSUPPORTED;
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
    if (err == cudaSuccess) err = cudaMalloc(&e->d_ref_end, std::max<uint64_t>(blocks, 1) * sizeof(RefEnd));
    if (err == cudaSuccess) err = cudaMalloc(&e->d_trans, std::max<uint64_t>(blocks, 1) * sizeof(BlockTrans));
    if (err == cudaSuccess) err = enc_upload(&e->d_block_seg, block_seg.data(), block_seg.size());
    if (err == cudaSuccess) err = enc_upload(&e->d_code_tab, code_tab.data(), code_tab.size());
    for (size_t i = 0; i < bounds.size(); ++i) {  // order keys (see order_key); a NaN bound: no level reached
      long long b;
      std::memcpy(&b, &bounds[i], 8);
      bound_keys[i] = std::isnan(bounds[i]) ? std::numeric_limits<long long>::max()
                                            : (b < 0 ? b ^ 0x7fffffffffffffffll : b);
    }
    if (err == cudaSuccess) err = enc_upload(&e->d_bound_keys, bound_keys.data(), bound_keys.size());
    e->w32 = true;
    for (uint32_t d = 0; d < n_domains; ++d) e->w32 = e->w32 && domains[d].N == 32 && domains[d].E == 16;
    if (err == cudaSuccess && e->w32) {  // the segment of each window kernel warp's first window
      const uint64_t per = 32u * kLvGroups, n = (win + per - 1) / per;
      std::vector<uint32_t> lvs(n);
      uint64_t sidx = 0;
      for (uint64_t c = 0; c < n; ++c) {
        const uint64_t g = c * per * 16u;  // its first level (E = 16)
        while (sidx + 1 < n_segments && segs[sidx + 1].level_offset <= g) ++sidx;
        lvs[c] = (uint32_t)sidx;
      }
      err = enc_upload(&e->d_lv_seg, lvs.data(), lvs.size());
    }
    if (err == cudaSuccess) err = cudaMalloc(&e->d_seg_bad, std::max<uint64_t>(n_segments, 1) * sizeof(uint32_t));
    // room for the bins decided in FP64: 0.2 % of them on signals, a few percent when
    // decoded signals are encoded again (their levels 127 and 129 reconstruct on the
    // deadzone edge); when it fills, the level kernels decide the rest themselves
    e->fb_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(lv / 16, 4096), uint64_t(1) << 28);
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
      if (enc->w32)
        k_enc_levels_w32<<<(unsigned)((enc->n_windows + kLvThreads * kLvGroups - 1) / (kLvThreads * kLvGroups)),
                           kLvThreads, 0, s>>>(p, enc->n_windows);
      else
        k_enc_levels<<<(unsigned)blocks, 256, 0, s>>>(p);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_enc_fallback<<<(unsigned)enc->sm_count * 8u, 256, 0, s>>>(p);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && enc->n_blocks) {
    k_enc_ref<<<(unsigned)((enc->n_blocks + 127) / 128), 128, 0, s>>>(p);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_enc_scan<<<(unsigned)((enc->n_segs * 32 + 127) / 128), 128, 0, s>>>(p);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && enc->n_blocks) {
    k_enc_pack<<<(unsigned)((enc->n_blocks + kPackWarps * 32 - 1) / (kPackWarps * 32)), kPackWarps * 32, 0, s>>>(p);
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
