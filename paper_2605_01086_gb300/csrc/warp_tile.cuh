// Shared machinery of the warp-tile decode kernels (FP32 transform in
// decode_warp.cu, tensor-core transform in decode_tc.cu), for the Table 1 shape
// N = 32, E = 16: tile constants, per-domain tables in shared memory, the
// SymLen word decoder, tile contexts and their asynchronous prefetch, the
// per-window dequantization, and the TMA store of 32-window output tiles.
// Included inside an anonymous namespace by each kernel file.
#pragma once

#include <cuda.h>

#include "device_util.cuh"

namespace fptc {
namespace wt {

constexpr int kN = 32;
constexpr int kE = 16;
constexpr int kT = 128;                    // windows per tile
constexpr int kTS = kT * kE;               // symbols per tile
constexpr int kGuard = 64;                 // entries before and after the tile (a word holds <= 64 codewords)
constexpr int kStage = kTS + 2 * kGuard;   // level bytes per warp
constexpr int kZStride = 257;              // floats per zone row (zero levels of the zones in different banks)
constexpr int kWPL = 2;                    // consecutive words per lane per decode pass
constexpr int kPassWords = 32 * kWPL;
constexpr int kStepWin = 32;               // windows per transform step (one per lane)
constexpr int kOutTile = kStepWin * kN * 4;  // bytes of a step's output (TMA box 32 x 32 floats)
constexpr int kMiscBytes = kPassWords * 8 + 32 + kStage;  // per warp: first-pass words, records, levels
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
__device__ __forceinline__ void tma_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct DomW {
  uint32_t lut_off;   // bytes from the start of shared memory: 16-bit entries len | level << 8
  uint32_t deq_off;   // bytes: zone rows [3][kZStride] floats (row 2 zero)
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
// codeword.  Returns error flags.
template <bool CHECKED>
__device__ __forceinline__ uint32_t decode_word(uint64_t w, uint32_t n, uint8_t *__restrict__ dst,
                                                const uint16_t *__restrict__ lut, uint32_t shift) {
  uint32_t hi = (uint32_t)(w >> 32), lo = (uint32_t)w, mk = 0x80000000u;
  uint32_t low = 31u;
  auto step = [&]() -> uint32_t {
    const uint32_t e = lut[hi >> shift];
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
  for (; j + 2 <= n; j += 2) {
    const uint32_t e0 = step();
    const uint32_t e1 = step();
    *reinterpret_cast<uint16_t *>(dst + j) = (uint16_t)__byte_perm(e0, e1, 0x0051);
  }
  if (j < n) dst[j] = (uint8_t)(step() >> 8);
  return ((hi | lo | mk) == 0u ? kFlagBitOverrun : 0u) | ((CHECKED && low == 0u) ? kFlagInvalidCode : 0u);
}

// Where a tile's words are (first word, count, codewords of the first word
// that belong to the previous tile) and its segment.
struct Ctx {
  uint64_t fw;
  uint32_t nw;
  uint32_t skip;
  uint32_t seg;
  uint32_t ok;  // 0: segment flagged by the index, or no tile
};

__device__ __forceinline__ Ctx make_ctx(const DecodeParams &p, uint64_t g, uint32_t s, const TileRec &r,
                                        const TileRec &rn) {
  Ctx c{0, 0, 0, s, 0};
  const SegDev &sg = p.segs[s];
  if (p.seg_bad[s] != 0) return c;
  const uint64_t tin = g - sg.tile_base;
  c.fw = r.first_word;
  c.skip = r.skip;
  uint64_t lw;
  if (tin + 1 < sg.n_tiles)
    lw = rn.first_word - (rn.skip == 0 ? 1u : 0u);
  else
    lw = sg.word_offset + sg.n_words - 1;
  c.nw = lw >= c.fw ? (uint32_t)(lw - c.fw + 1) : 0u;
  c.ok = 1;
  return c;
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

// Records of tiles g and g + 1 into rec[0..1] (lanes 0 and 1).
__device__ __forceinline__ void fetch_records(const DecodeParams &p, uint64_t g, uint32_t lane, TileRec *rec) {
  if (lane < 2 && g + lane < p.tile_end) cp_async16(rec + lane, p.tiles + g + lane);
  cp_async_commit();
}

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
    off = deq_off + (uint32_t)align16(3u * kZStride * 4);
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
    for (uint32_t i = threadIdx.x; i < 3u * kZStride; i += THREADS) {
      const uint32_t z = i / kZStride, L = i - z * kZStride;
      deq[i] = (L < 256u && z < 2u) ? (z == 0 ? a0 : a1) * dm.unit[z][L] : 0.0f;
    }
  }
  return off;
}

// SymLen decode of one tile (Sec. 4.2.1) into the level bytes at stage[0..):
// passes of two consecutive words per lane, a warp scan of their symbol
// counts, the codewords of each word at their tile positions (those of the
// previous tile, and after the tile's last symbol, go to the guards).  w/n
// hold the first pass's words; later passes are loaded one pass ahead.
// Returns the OR of the error flags over the warp.
__device__ __forceinline__ uint32_t decode_tile(const DecodeParams &p, const Ctx &cur, const DomW &dd,
                                                const unsigned char *smem, uint8_t *stage, uint32_t lane,
                                                uint64_t (&w)[kWPL], uint32_t (&n)[kWPL]) {
  const uint16_t *lut = reinterpret_cast<const uint16_t *>(smem + dd.lut_off);
  int32_t base = -(int32_t)cur.skip;
  uint32_t bad = 0;
  for (uint32_t c0 = 0; c0 < cur.nw; c0 += kPassWords) {
    uint64_t xw[kWPL];
    uint32_t xn[kWPL];
    if (c0 + kPassWords < cur.nw) {
      load_pass(p, cur, c0 + kPassWords, lane, xw, xn);
    } else {
#pragma unroll
      for (int u = 0; u < kWPL; ++u) {
        xw[u] = 0;
        xn[u] = 0;
      }
    }
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
    uint8_t *dst = stage + base + (int32_t)(x - tot);
    if (dd.complete) {
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
    base += (int32_t)total;
#pragma unroll
    for (int u = 0; u < kWPL; ++u) {
      w[u] = xw[u];
      n[u] = xn[u];
    }
  }
  return __reduce_or_sync(0xffffffffu, bad);
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
    for (int k = 0; k < 16; ++k)
      c[k] = deq[((zmask >> (2 * k)) & 3u) * kZStride + ((sw[k >> 2] >> (8 * (k & 3))) & 0xffu)];
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
