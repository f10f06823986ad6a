// Shared machinery of the warp-tile decode kernels (FP32 transform in
// decode_warp.cu, tensor-core transform in decode_tc.cu), for the Table 1 shape
// N = 32, E = 16: tile constants, per-domain tables in shared memory, the
// SymLen word decoder, tile contexts and their asynchronous prefetch, the
// per-window dequantization, and the TMA store of 32-window output tiles.
//
// Each warp decodes a contiguous range of tiles.  The first tile of the range
// is located from the index's chunk offsets (symbol_word); every later tile of
// a segment starts at the word where the tile before it ended, which the SymLen
// decode of that tile finds anyway, so no record per tile is read.
#pragma once

#include <cuda.h>

#include "device_util.cuh"
#include "symlen_chunks.cuh"

namespace fptc {
namespace wt {

constexpr int kN = 32;
constexpr int kE = 16;
constexpr int kT = 128;                    // windows per tile
constexpr int kTS = kT * kE;               // symbols per tile
constexpr int kGuard = 64;                 // entries before and after the tile (a word holds <= 64 codewords)
constexpr int kStage = kTS + kGuard;       // level bytes per warp after the first-pass words (see kStageOff)
constexpr int kZStride = 257;              // floats per zone row (zero levels of the zones in different banks)
constexpr int kZRows = 2;                  // zone rows in shared memory: zone 2 reconstructs 0 without a row
constexpr uint32_t kDeqBytes = (kZRows * kZStride * 4 + 15) / 16 * 16;  // a domain's dequantization rows
constexpr int kWPL = 2;                    // consecutive words per lane per decode pass
constexpr int kPassWords = 32 * kWPL;
constexpr int kStepWin = 32;               // windows per transform step (one per lane)
constexpr int kOutTile = kStepWin * kN * 4;  // bytes of a step's output (TMA box 32 x 32 floats)
// Per warp: the first-pass words, then the level bytes.  The guard before tile
// position 0 is the last kGuard bytes of the first-pass words: those words are
// in registers before the decode writes there, and the next tile's words are
// requested only after it (decode_tile ends with a warp barrier).
constexpr int kMiscBytes = kPassWords * 8 + kStage;
constexpr int kStageOff = kPassWords * 8;  // tile position 0 from the start of the warp's area
static_assert(kGuard <= kPassWords * 8, "the guard before the tile lies inside the first-pass words");
static_assert(kStageOff % 16 == 0 && kMiscBytes % 16 == 0, "level rows are read as 16-byte vectors");
// zone mask of Table 1 (B1 = 2, B2 = 16): bins 0, 1 in zone 0, the rest in zone 1
constexpr uint32_t kZmaskTable1 = 0x55555550u;

// 32-byte streaming store (one full sector per thread)
__device__ __forceinline__ void st_cs_v8(float *p, const float (&v)[8]) {
  asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}

// TMA tensor store of a staged 32 x 32-float tile to rows [row, row + 32) of
// the output, and the waits on it (bulk async-group of the issuing thread).
__device__ __forceinline__ void tma_store_rows(const CUtensorMap *map, const void *smem_tile, int32_t row) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(0), "r"(row), "r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem_tile)))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// ---- bounded mbarrier waits ---------------------------------------------------
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
// One test of the phase of parity `parity`; the thread may be suspended up to
// hint_ns until that phase completes (it does not spin meanwhile).
__device__ __forceinline__ bool mbar_try_wait_for(uint32_t addr, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
constexpr uint64_t kWaitNs = 1000000000ull;  // a wait gives up after 1 s of global time
// Waits for the phase of parity `parity` of the mbarrier at addr, sleeping in
// try_wait between tests; false if it has not completed after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  if (mbar_try_wait_for(addr, parity, 20000u)) return true;
  const uint64_t t0 = global_ns();
  do {
    if (mbar_try_wait_for(addr, parity, 1000000u)) return true;
  } while (global_ns() - t0 < kWaitNs);
  return false;
}

__device__ __forceinline__ void tma_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct DomW {
  uint32_t lut_off;   // bytes from the start of shared memory: 16-bit entries len | level << 8
  uint32_t deq_off;   // bytes: zone rows [kZRows][kZStride] floats (zones 0 and 1)
  uint32_t shift;     // 32 - lmax
  uint32_t zmask;     // zone of bin k at bits 2k..2k+1
  uint32_t complete;  // every prefix decodes (no zero entry)
  uint32_t pad[3];
};

// Codewords of one SymLen word, MSB first.  w's bits sit in hi:lo with a marker
// bit right under them (mk); each codeword shifts the 96 bits left by its
// length (the entry's low 5 bits: the funnel shifts use the amount mod 32).
// The marker leaves the buffer iff the codewords used more than 64 bits.
// CHECKED (incomplete code): an entry of length 0 marks a prefix with no
// codeword.  SHIFT: 32 - lmax when the caller knows it at compile time (the
// table index is then one shift-and-add), else 0 and `shift` holds it.
// Returns error flags.
template <bool CHECKED, uint32_t SHIFT = 0>
__device__ __forceinline__ uint32_t decode_word(uint64_t w, uint32_t n, uint8_t *__restrict__ dst,
                                                const uint16_t *__restrict__ lut, uint32_t shift) {
  uint32_t hi = (uint32_t)(w >> 32), lo = (uint32_t)w, mk = 0x80000000u;
  uint32_t low = 31u;
  auto step = [&]() -> uint32_t {
    const uint32_t e = lut[hi >> (SHIFT ? SHIFT : shift)];
    hi = __funnelshift_l(lo, hi, e);
    lo = __funnelshift_l(mk, lo, e);
    mk = __funnelshift_l(0u, mk, e);
    if (CHECKED) low = min(low, e & 31u);
    return e;
  };
  // levels go out two per 16-bit store where both are this word's
  uint32_t j = 0;
  if (n && (reinterpret_cast<uintptr_t>(dst) & 1u)) {
    dst[0] = (uint8_t)(step() >> 8);
    j = 1;
  }
  for (; j + 4 <= n; j += 4) {  // four codewords an iteration (less loop overhead per codeword)
    const uint32_t e0 = step();
    const uint32_t e1 = step();
    const uint32_t e2 = step();
    const uint32_t e3 = step();
    *reinterpret_cast<uint16_t *>(dst + j) = (uint16_t)__byte_perm(e0, e1, 0x0051);
    *reinterpret_cast<uint16_t *>(dst + j + 2) = (uint16_t)__byte_perm(e2, e3, 0x0051);
  }
  if (j + 2 <= n) {
    const uint32_t e0 = step();
    const uint32_t e1 = step();
    *reinterpret_cast<uint16_t *>(dst + j) = (uint16_t)__byte_perm(e0, e1, 0x0051);
    j += 2;
  }
  if (j < n) dst[j] = (uint8_t)(step() >> 8);
  return ((hi | lo | mk) == 0u ? kFlagBitOverrun : 0u) | ((CHECKED && low == 0u) ? kFlagInvalidCode : 0u);
}

// Where a tile's words are (first word, words that may belong to it, codewords
// of the first word that belong to the previous tile) and its segment.
struct Ctx {
  uint64_t fw;
  uint32_t nw;
  uint32_t skip;
  uint32_t seg;
  uint32_t ok;  // 0: segment flagged by the index, or no tile
};

// Context of a tile of segment s starting at word fw after `skip` symbols.  A
// tile holds at most kTS symbols and every word of a valid stream at least
// one, so it spans at most kTS + 1 words (fewer at the segment's end).
__device__ __forceinline__ Ctx make_ctx(const DecodeParams &p, uint32_t s, uint64_t fw, uint32_t skip) {
  Ctx c{fw, 0, skip, s, 0};
  if (p.seg_bad[s] != 0) return c;
  const SegDev &sg = p.segs[s];
  const uint64_t end = sg.word_offset + sg.n_words;
  c.nw = fw < end ? (uint32_t)min(end - fw, (uint64_t)kTS + 1u) : 0u;
  c.ok = 1;
  return c;
}

// Context of tile g of segment s (tiles of tile_syms symbols) located from the
// index (warp-collective).
__device__ __forceinline__ Ctx first_ctx(const DecodeParams &p, uint32_t s, uint64_t g, uint32_t lane,
                                         uint64_t tile_syms = kTS) {
  const SegDev &sg = p.segs[s];
  if (p.seg_bad[s] != 0) return Ctx{0, 0, 0, s, 0};
  const uint64_t tin = g - sg.tile_base;
  if (tin == 0) return make_ctx(p, s, sg.word_offset, 0u);
  const TileRec r = symbol_word(p.symlen, p.chunk_off, sg, tin * tile_syms, lane);
  if (r.pad != 0) return Ctx{0, 0, 0, s, 0};
  return make_ctx(p, s, r.first_word, r.skip);
}

// Where a decoded tile ended: the word (from the tile's first word) holding
// the next tile's first symbol and the symbols of it that were this tile's.
struct TileEnd {
  uint32_t bad;  // error flags (OR over the warp)
  uint32_t word;
  uint32_t skip;
};

// Context of tile g + 1 after tile g (segment s, context cur) ended at e.
__device__ __forceinline__ Ctx next_ctx(const DecodeParams &p, uint64_t g, uint32_t s, const Ctx &cur,
                                        const TileEnd &e) {
  if (g + 1 < p.segs[s].tile_base + p.segs[s].n_tiles) {
    if (!cur.ok) return Ctx{0, 0, 0, s, 0};
    return make_ctx(p, s, cur.fw + e.word, e.skip);
  }
  uint32_t s1 = s + 1;
  while (g + 1 >= p.segs[s1].tile_base + p.segs[s1].n_tiles) ++s1;  // segments without tiles
  return make_ctx(p, s1, p.segs[s1].word_offset, 0u);
}

// Words i0 + kWPL lane + u (u < kWPL) of a tile (zero beyond its word count).
__device__ __forceinline__ void load_pass(const DecodeParams &p, const Ctx &c, uint32_t i0, uint32_t lane,
                                          uint64_t (&w)[kWPL], uint32_t (&n)[kWPL]) {
#pragma unroll
  for (int u = 0; u < kWPL; ++u) {
    const uint32_t i = i0 + kWPL * lane + u;
    const bool in = c.ok && i < c.nw;
    w[u] = in ? __ldg(p.words + c.fw + i) : 0ull;
    n[u] = in ? (uint32_t)__ldg(p.symlen + c.fw + i) : 0u;
  }
}

__device__ __forceinline__ uint32_t smem_addr(const void *ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

// Asynchronous global -> shared copies (no register staging; completion by
// cp.async.wait_all in the copying thread).
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// First pass of a tile: words kWPL lane + u into wbuf (copies), their symbol
// counts packed one per byte into a register (zero beyond the tile's words).
__device__ __forceinline__ uint32_t fetch_pass0(const DecodeParams &p, const Ctx &c, uint32_t lane, uint64_t *wbuf) {
  uint32_t packed = 0;
#pragma unroll
  for (int u = 0; u < kWPL; ++u) {
    const uint32_t i = kWPL * lane + u;
    if (c.ok && i < c.nw) {
      cp_async8(wbuf + i, p.words + c.fw + i);
      packed |= (uint32_t)__ldg(p.symlen + c.fw + i) << (8 * u);
    }
  }
  cp_async_commit();
  return packed;
}

// Every domain's tables into shared memory from byte 0 (the layout of
// warp_smem_layout; offsets computed here, not indexed from a parameter
// block): the DomW array, then per domain the decode table (entries rewritten
// len | level << 8) and the dequantization rows.  Returns the end offset.
// Contains no barrier.
template <int THREADS>
__device__ __forceinline__ uint32_t load_domain_tables(const DecodeParams &p, uint32_t n_domains, unsigned char *smem) {
  DomW *const dw = reinterpret_cast<DomW *>(smem);
  uint32_t off = (uint32_t)align16(sizeof(DomW) * (n_domains ? n_domains : 1));
  for (uint32_t d = 0; d < n_domains; ++d) {
    const DomainDev &dm = p.domains[d];
    const uint32_t lut_off = off;
    const uint32_t deq_off = lut_off + (uint32_t)align16((size_t)2 << dm.lmax);
    off = deq_off + kDeqBytes;
    if (threadIdx.x == 0) {
      DomW x;
      x.lut_off = lut_off;
      x.deq_off = deq_off;
      x.shift = 32u - dm.lmax;
      uint32_t zm = 0;
      for (uint32_t k = 0; k < kE; ++k) zm |= (k < dm.B1 ? 0u : (k < dm.B2 ? 1u : 2u)) << (2 * k);
      x.zmask = zm;
      x.complete = dm.complete;
      x.pad[0] = x.pad[1] = x.pad[2] = 0;
      dw[d] = x;
    }
    uint16_t *lut = reinterpret_cast<uint16_t *>(smem + lut_off);
    const uint16_t *g_lut = p.luts + dm.lut_offset;
    const uint32_t entries = 1u << dm.lmax;
    for (uint32_t i = threadIdx.x; i < entries; i += THREADS) {
      const uint32_t v = __ldg(g_lut + i);
      lut[i] = (uint16_t)((v >> 8) | ((v & 0xffu) << 8));
    }
    float a0 = p.scale ? p.scale[d * 3 + 0] : dm.scale[0];
    float a1 = p.scale ? p.scale[d * 3 + 1] : dm.scale[1];
    a0 = a0 > 1e-30f ? a0 : 0.0f;
    a1 = a1 > 1e-30f ? a1 : 0.0f;
    float *deq = reinterpret_cast<float *>(smem + deq_off);
    for (uint32_t i = threadIdx.x; i < (uint32_t)(kZRows * kZStride); i += THREADS) {
      const uint32_t z = i / kZStride, L = i - z * kZStride;
      deq[i] = L < 256u ? (z == 0 ? a0 : a1) * dm.unit[z][L] : 0.0f;
    }
  }
  return off;
}

// SymLen decode of one tile of `te` symbols (Sec. 4.2.1) into the level bytes
// at stage[0..): passes of two consecutive words per lane, a warp scan of their
// symbol counts, the codewords of each word at their tile positions (those of
// the previous tile go to the guard before the tile, those after the tile's
// last symbol to the guard after it).  The pass whose scan reaches te is the
// last: its words that start at or after te are left to the next tile, and the
// word holding symbol te is where the next tile starts.  w/n hold the first
// pass's words; each later pass is loaded while the one before it decodes.
// D: the domain's table view (lut_off, shift, complete).
template <class D>
__device__ __forceinline__ TileEnd decode_tile(const DecodeParams &p, const Ctx &cur, uint32_t te, const D &dd,
                                               const unsigned char *smem, uint8_t *stage, uint32_t lane,
                                               uint64_t (&w)[kWPL], uint32_t (&n)[kWPL]) {
  const uint16_t *lut = reinterpret_cast<const uint16_t *>(smem + dd.lut_off);
  int32_t base = -(int32_t)cur.skip;
  uint32_t bad = 0;
  TileEnd r{0u, 0u, 0u};
  for (uint32_t c0 = 0; c0 < cur.nw; c0 += kPassWords) {
    uint32_t tot = 0;
#pragma unroll
    for (int u = 0; u < kWPL; ++u) tot += n[u];
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    const int32_t p0 = base + (int32_t)(x - tot);  // tile position of this lane's first symbol
    const bool last = base + (int32_t)total >= (int32_t)te;
    uint64_t xw[kWPL];
    uint32_t xn[kWPL];
    if (!last && c0 + kPassWords < cur.nw) {
      load_pass(p, cur, c0 + kPassWords, lane, xw, xn);
    } else {
#pragma unroll
      for (int u = 0; u < kWPL; ++u) {
        xw[u] = 0;
        xn[u] = 0;
      }
    }
    if (last) {
      uint32_t hit = 0u, hw = 0u, hs = 0u;
      int32_t q = p0;
#pragma unroll
      for (int u = 0; u < kWPL; ++u) {
        const int32_t qe = q + (int32_t)n[u];
        if (!hit && q <= (int32_t)te && (int32_t)te < qe) {
          hit = 1u;
          hw = c0 + kWPL * lane + u;
          hs = (uint32_t)((int32_t)te - q);
        }
        if (q >= (int32_t)te) n[u] = 0u;
        q = qe;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, hit);
      if (m) {
        const uint32_t src = (uint32_t)(__ffs(m) - 1);
        r.word = __shfl_sync(0xffffffffu, hw, src);
        r.skip = __shfl_sync(0xffffffffu, hs, src);
      } else {  // the tile ends with this pass's last word
        r.word = c0 + kPassWords;
        r.skip = 0u;
      }
    }
    uint8_t *dst = stage + p0;
    if (dd.complete && dd.shift == 20u) {  // L_max = 12, the trained tables' limit
#pragma unroll
      for (int u = 0; u < kWPL; ++u) {
        bad |= decode_word<false, 20u>(w[u], n[u], dst, lut, 20u);
        dst += n[u];
      }
    } else if (dd.complete) {
#pragma unroll
      for (int u = 0; u < kWPL; ++u) {
        bad |= decode_word<false>(w[u], n[u], dst, lut, dd.shift);
        dst += n[u];
      }
    } else {
#pragma unroll
      for (int u = 0; u < kWPL; ++u) {
        bad |= decode_word<true>(w[u], n[u], dst, lut, dd.shift);
        dst += n[u];
      }
    }
    if (last) break;
    base += (int32_t)total;
#pragma unroll
    for (int u = 0; u < kWPL; ++u) {
      w[u] = xw[u];
      n[u] = xn[u];
    }
  }
  r.bad = __reduce_or_sync(0xffffffffu, bad);
  __syncwarp();  // the guard before the tile is the first-pass words' area, refilled after this
  return r;
}

// The 16 coefficients A_z * unit_z(level) of a window from its 16 level bytes
// (Eq. 2 / Eq. 3 inverted by table: one shared-memory read per bin).
__device__ __forceinline__ void window_coefs(const uint4 &sv, const float *deq, uint32_t zmask, float (&c)[16]) {
  const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w};
  if (zmask == kZmaskTable1) {
#pragma unroll
    for (int k = 0; k < 16; ++k) c[k] = deq[(k < 2 ? 0 : kZStride) + ((sw[k >> 2] >> (8 * (k & 3))) & 0xffu)];
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t z = (zmask >> (2 * k)) & 3u;
      c[k] = z < 2u ? deq[z * kZStride + ((sw[k >> 2] >> (8 * (k & 3))) & 0xffu)] : 0.0f;  // zone 2: 0
    }
  }
}

// The window's levels to the caller's level buffer (16 bytes).
__device__ __forceinline__ void put_levels(uint8_t *dl, const uint4 &sv) {
  if ((reinterpret_cast<uintptr_t>(dl) & 15u) == 0) {
    *reinterpret_cast<uint4 *>(dl) = sv;
  } else {
    const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) dl[j] = (uint8_t)(sw[j >> 2] >> (8 * (j & 3)));
  }
}

// A row of 32 samples from the staging tile (16-byte chunk c at c ^ (row & 7),
// sx = row & 7) to dst: m samples, 32-byte or 16-byte streaming stores where
// the alignment allows.
__device__ __forceinline__ void store_row(const unsigned char *row, uint32_t sx, float *dst, uint32_t m, bool vec32,
                                          bool vec16) {
  if (m == 32 && (vec32 || vec16)) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float4 u = *reinterpret_cast<const float4 *>(row + (((2 * b) ^ sx) << 4));
      const float4 v = *reinterpret_cast<const float4 *>(row + (((2 * b + 1) ^ sx) << 4));
      if (vec32) {
        const float x[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
        st_cs_v8(dst + 8 * b, x);
      } else {
        __stcs(reinterpret_cast<float4 *>(dst + 8 * b), u);
        __stcs(reinterpret_cast<float4 *>(dst + 8 * b) + 1, v);
      }
    }
  } else {
    for (uint32_t n = 0; n < m; ++n)
      dst[n] = *reinterpret_cast<const float *>(row + ((((n >> 2) ^ sx) << 4) | ((n & 3u) << 2)));
  }
}

// The warp's tile range of a launch, for tiles handed out `per` at a time to
// `units` units (warps, or warpgroups of `per` warps).
__device__ __forceinline__ void unit_tiles(const DecodeParams &p, uint64_t unit, uint64_t units, uint64_t &t0,
                                           uint64_t &t1) {
  const uint64_t n_all = p.tile_end - p.tile_begin;
  t0 = p.tile_begin + n_all * unit / units;
  t1 = p.tile_begin + n_all * (unit + 1) / units;
}

}  // namespace wt
}  // namespace fptc
