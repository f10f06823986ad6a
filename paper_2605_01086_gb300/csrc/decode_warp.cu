// Fused decode for the Table 1 shape (N = 32, E = 16) with one warp per tile.
//
// Each warp owns a contiguous range of tiles of 64 windows (1024 symbols, 2048
// samples) and runs Sec. 4.2 on each with no block-wide barrier:
//  1. SymLen decode.  A pass gives every lane two consecutive words; a warp
//     scan of their symbol counts places each word's codewords (compaction,
//     Sec. 4.2.1).  A lane decodes a word with one decode-table lookup per
//     codeword and stores the table entry (code length | level << 8) as a
//     16-bit value at the codeword's tile position.  Nothing else happens per
//     codeword: the dequantization waits for step 2, where the bin of every
//     value is known at compile time.  The 64-bit word is shifted through
//     hi:lo with a marker bit under it, so a word whose codewords need more
//     than 64 bits shows as an empty buffer at the end (no per-codeword count).
//  2. Dequantization and inverse DCT in steps of 16 windows.  Lane (r, q)
//     turns bins 4q..4q+3 of windows r and r+8 into A_z * unit_z(level) (one
//     table read each) and writes them to a padded row buffer; after a
//     __syncwarp the four lanes of a window read its 16 coefficients and
//     compute 4 samples and their 4 mirror samples with FFMA2 (even/odd bin
//     pairs, B[k][N-1-n] = (-1)^k B[k][n]); 16-byte streaming stores.
//  The tile records of tile g+1 are loaded when tile g starts, the first words
//  of tile g+1 when tile g's decode ends (hidden by its transform), and the
//  words of a tile's next decode pass before the current pass.
// The decode tables, dequantization rows and basis of every domain stay in
// shared memory for the whole kernel.
#include "device_util.cuh"

namespace fptc {
namespace {

constexpr int kN = 32;
constexpr int kE = 16;
constexpr int kT = 64;                     // windows per tile
constexpr int kTS = kT * kE;               // symbols per tile
constexpr int kGuard = 64;                 // entries before and after the tile (a word holds <= 64 codewords)
constexpr int kStage = kTS + 2 * kGuard;   // 16-bit entries per warp
constexpr int kZStride = 257;              // floats per zone row (zero levels of the zones in different banks)
constexpr int kStepWin = 16;               // windows per transform step
constexpr int kRowF = 20;                  // floats per coefficient row: 8 rows read at once hit 8 bank groups
constexpr int kWPL = 2;                    // words per lane per decode pass
constexpr int kPassWords = 32 * kWPL;

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
__device__ __forceinline__ uint32_t decode_word(uint64_t w, uint32_t n, uint16_t *__restrict__ dst,
                                                const uint16_t *__restrict__ lut, uint32_t shift) {
  uint32_t hi = (uint32_t)(w >> 32), lo = (uint32_t)w, mk = 0x80000000u;
  uint32_t low = 31u;
  for (uint32_t j = 0; j < n; ++j) {
    const uint32_t e = lut[hi >> shift];
    hi = __funnelshift_l(lo, hi, e);
    lo = __funnelshift_l(mk, lo, e);
    mk = __funnelshift_l(0u, mk, e);
    dst[j] = (uint16_t)e;
    if (CHECKED) low = min(low, e & 31u);
  }
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

// Words i0 + 2 lane, i0 + 2 lane + 1 of a tile (zero beyond its word count).
__device__ __forceinline__ void load_pass(const DecodeParams &p, const Ctx &c, uint32_t i0, uint32_t lane,
                                          uint64_t &wa, uint64_t &wb, uint32_t &na, uint32_t &nb) {
  const uint32_t i = i0 + 2 * lane;
  const bool ia = c.ok && i < c.nw, ib = c.ok && i + 1 < c.nw;
  wa = ia ? __ldg(p.words + c.fw + i) : 0ull;
  wb = ib ? __ldg(p.words + c.fw + i + 1) : 0ull;
  na = ia ? (uint32_t)__ldg(p.symlen + c.fw + i) : 0u;
  nb = ib ? (uint32_t)__ldg(p.symlen + c.fw + i + 1) : 0u;
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

// First pass of a tile: words 2 lane, 2 lane + 1 into wbuf (copies), their
// symbol counts into registers (zero beyond the tile's words).
__device__ __forceinline__ void fetch_pass0(const DecodeParams &p, const Ctx &c, uint32_t lane, uint64_t *wbuf,
                                            uint32_t &na, uint32_t &nb) {
  const uint32_t i = 2 * lane;
  const bool ia = c.ok && i < c.nw, ib = c.ok && i + 1 < c.nw;
  if (ia) cp_async8(wbuf + i, p.words + c.fw + i);
  if (ib) cp_async8(wbuf + i + 1, p.words + c.fw + i + 1);
  cp_async_commit();
  na = ia ? (uint32_t)__ldg(p.symlen + c.fw + i) : 0u;
  nb = ib ? (uint32_t)__ldg(p.symlen + c.fw + i + 1) : 0u;
}

__device__ __forceinline__ void store_window(float *out, uint64_t S, uint64_t s0, uint32_t q, const float2 (&acc)[4],
                                             uint32_t aligned) {
  const float4 lo = make_float4(acc[0].x + acc[0].y, acc[1].x + acc[1].y, acc[2].x + acc[2].y, acc[3].x + acc[3].y);
  const float4 hi = make_float4(acc[3].x - acc[3].y, acc[2].x - acc[2].y, acc[1].x - acc[1].y, acc[0].x - acc[0].y);
  float *dst = out + s0;
  if (s0 + kN <= S && aligned) {
    __stcs(reinterpret_cast<float4 *>(dst + 4 * q), lo);
    __stcs(reinterpret_cast<float4 *>(dst + kN - 4 - 4 * q), hi);
  } else {
    const float lv[4] = {lo.x, lo.y, lo.z, lo.w};
    const float hv[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t n1 = 4 * q + j, n2 = kN - 4 - 4 * q + j;
      if (s0 + n1 < S) dst[n1] = lv[j];
      if (s0 + n2 < S) dst[n2] = hv[j];
    }
  }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS) k_decode_warp(const DecodeParams p,
                                                                                 const WarpParams wp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DomW *const dw = reinterpret_cast<DomW *>(smem_raw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // ---- every domain's tables, once (offsets as in warp_smem_layout; computed
  // here rather than indexed from the parameter block)
  uint32_t off = (uint32_t)align16(sizeof(DomW) * (wp.n_domains ? wp.n_domains : 1));
  for (uint32_t d = 0; d < wp.n_domains; ++d) {
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
    // entries level | len << 8 -> len | level << 8 (the length in the low bits feeds the shifts)
    uint16_t *lut = reinterpret_cast<uint16_t *>(smem_raw + lut_off);
    const uint16_t *g_lut = p.luts + dm.lut_offset;
    const uint32_t entries = 1u << dm.lmax;
    for (uint32_t i = threadIdx.x; i < entries; i += WARPS * 32) {
      const uint32_t v = __ldg(g_lut + i);
      lut[i] = (uint16_t)((v >> 8) | ((v & 0xffu) << 8));
    }
    float a0 = p.scale ? p.scale[d * 3 + 0] : dm.scale[0];
    float a1 = p.scale ? p.scale[d * 3 + 1] : dm.scale[1];
    a0 = a0 > 1e-30f ? a0 : 0.0f;
    a1 = a1 > 1e-30f ? a1 : 0.0f;
    float *deq = reinterpret_cast<float *>(smem_raw + deq_off);
    for (uint32_t i = threadIdx.x; i < 3u * kZStride; i += WARPS * 32) {
      const uint32_t z = i / kZStride, L = i - z * kZStride;
      deq[i] = (L < 256u && z < 2u) ? (z == 0 ? a0 : a1) * dm.unit[z][L] : 0.0f;
    }
  }
  {
    // paired basis (B[2m][n], B[2m+1][n]), [m][n]; the same for every N = 32, E = 16 domain
    float2 *bp = reinterpret_cast<float2 *>(smem_raw + wp.basis_off);
    const float *b = p.basis + p.domains[0].basis_offset;
    for (uint32_t i = threadIdx.x; i < (kE / 2) * kN; i += WARPS * 32) {
      const uint32_t m = i / kN, n = i % kN;
      bp[i] = make_float2(__ldg(b + (2 * m) * kN + n), __ldg(b + (2 * m + 1) * kN + n));
    }
  }
  __syncthreads();

  unsigned char *const wbase = smem_raw + wp.warp_off + warp * wp.warp_bytes;
  uint64_t *const wbuf = reinterpret_cast<uint64_t *>(wbase);                       // first-pass words
  TileRec *const rec = reinterpret_cast<TileRec *>(wbase + kPassWords * 8);          // records g, g + 1
  uint16_t *const stage = reinterpret_cast<uint16_t *>(wbase + kPassWords * 8 + 32) + kGuard;  // tile position 0
  float *const cbuf0 = reinterpret_cast<float *>(wbase + kPassWords * 8 + 32 + kStage * 2);
  float *const cbuf1 = cbuf0 + kStepWin * kRowF;
  const float4 *const bas4 = reinterpret_cast<const float4 *>(smem_raw + wp.basis_off);  // [m][16]
  const bool want_lev = p.levels != nullptr;
  const uint32_t r = lane >> 2, q = lane & 3u;

  // ---- this warp's tiles: an even split of the launch's tile range over all warps
  const uint64_t n_all = p.tile_end - p.tile_begin;
  const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
  const uint64_t gw = (uint64_t)blockIdx.x * WARPS + warp;
  const uint64_t tw0 = p.tile_begin + n_all * gw / nwarps;
  const uint64_t tw1 = p.tile_begin + n_all * (gw + 1) / nwarps;
  if (tw0 >= tw1) return;

  // prologue: records of tw0, then its first words
  uint32_t s = find_segment(p.segs, p.seg_begin, p.seg_end, tw0);
  fetch_records(p, tw0, lane, rec);
  cp_async_wait_all();
  __syncwarp();
  uint32_t pna, pnb;
  fetch_pass0(p, make_ctx(p, tw0, s, rec[0], rec[1]), lane, wbuf, pna, pnb);

  for (uint64_t g = tw0; g < tw1; ++g) {
    // ---- tile g: its records and first words have been requested
    cp_async_wait_all();
    __syncwarp();
    while (g >= p.segs[s].tile_base + p.segs[s].n_tiles) ++s;
    const Ctx cur = make_ctx(p, g, s, rec[0], rec[1]);
    uint64_t wa = wbuf[2 * lane], wb = wbuf[2 * lane + 1];
    uint32_t na = pna, nb = pnb;
    __syncwarp();
    const uint64_t g1 = g + 1;
    if (g1 < tw1) fetch_records(p, g1, lane, rec);  // consumed after the decode

    const SegDev &sg = p.segs[cur.seg];
    const uint32_t dom = sg.domain;
    const DomW dd = dw[dom];
    const uint64_t win0 = (g - sg.tile_base) * kT;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = left < (uint64_t)kT ? (uint32_t)left : (uint32_t)kT;

    // ---- 1. SymLen decode into the staging entries
    if (cur.ok) {
      const uint16_t *lut = reinterpret_cast<const uint16_t *>(smem_raw + dd.lut_off);
      int32_t base = -(int32_t)cur.skip;
      uint32_t bad = 0;
      for (uint32_t c0 = 0; c0 < cur.nw; c0 += kPassWords) {
        uint64_t xa = 0, xb = 0;
        uint32_t xna = 0, xnb = 0;
        if (c0 + kPassWords < cur.nw) load_pass(p, cur, c0 + kPassWords, lane, xa, xb, xna, xnb);
        const uint32_t tot = na + nb;
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= (uint32_t)o) x += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
        uint16_t *dst = stage + base + (int32_t)(x - tot);
        if (dd.complete) {
          bad |= decode_word<false>(wa, na, dst, lut, dd.shift);
          bad |= decode_word<false>(wb, nb, dst + na, lut, dd.shift);
        } else {
          bad |= decode_word<true>(wa, na, dst, lut, dd.shift);
          bad |= decode_word<true>(wb, nb, dst + na, lut, dd.shift);
        }
        base += (int32_t)total;
        wa = xa;
        wb = xb;
        na = xna;
        nb = xnb;
      }
      bad = __reduce_or_sync(0xffffffffu, bad);
      if (bad && lane == 0) flag_bad(p.status, bad, sg.caller_index);
    }

    // ---- first words of tile g + 1 (in flight during the transform)
    if (g1 < tw1) {
      cp_async_wait_all();
      __syncwarp();
      uint32_t s1 = s;
      while (g1 >= p.segs[s1].tile_base + p.segs[s1].n_tiles) ++s1;
      fetch_pass0(p, make_ctx(p, g1, s1, rec[0], rec[1]), lane, wbuf, pna, pnb);
    }
    __syncwarp();

    // ---- 2. dequantization + inverse transform + reassembly, 16 windows per step
    if (cur.ok) {
      const float *deq = reinterpret_cast<const float *>(smem_raw + dd.deq_off);
      const float *row0 = deq + ((dd.zmask >> (8 * q + 0)) & 3u) * kZStride;
      const float *row1 = deq + ((dd.zmask >> (8 * q + 2)) & 3u) * kZStride;
      const float *row2 = deq + ((dd.zmask >> (8 * q + 4)) & 3u) * kZStride;
      const float *row3 = deq + ((dd.zmask >> (8 * q + 6)) & 3u) * kZStride;
      float *const out = p.out + sg.out_offset;
      const uint64_t S = sg.n_samples;
      const uint32_t aligned = sg.out_aligned;
      uint8_t *const lev = want_lev ? p.levels + sg.level_offset + win0 * kE : nullptr;
#pragma unroll 1
      for (uint32_t w0 = 0; w0 < nwin; w0 += kStepWin) {
        float *const cb = (w0 & kStepWin) ? cbuf1 : cbuf0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t w = w0 + r + 8 * h;
          const uint2 ev = *reinterpret_cast<const uint2 *>(stage + w * kE + 4 * q);
          float4 c;
          c.x = row0[(ev.x >> 8) & 0xffu];
          c.y = row1[ev.x >> 24];
          c.z = row2[(ev.y >> 8) & 0xffu];
          c.w = row3[ev.y >> 24];
          *reinterpret_cast<float4 *>(cb + (r + 8 * h) * kRowF + 4 * q) = c;
          if (want_lev && w < nwin) {
            const uint32_t l4 = __byte_perm(ev.x, ev.y, 0x7531);
            uint8_t *dl = lev + w * kE + 4 * q;
            if ((reinterpret_cast<uintptr_t>(dl) & 3u) == 0) {
              *reinterpret_cast<uint32_t *>(dl) = l4;
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j) dl[j] = (uint8_t)(l4 >> (8 * j));
            }
          }
        }
        __syncwarp();
        const uint32_t wa = w0 + r, wb = wa + 8;
        if (wa < nwin) {
          const float4 *ca = reinterpret_cast<const float4 *>(cb + r * kRowF);
          const float4 *cbv = reinterpret_cast<const float4 *>(cb + (r + 8) * kRowF);
          float2 accA[4], accB[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) accA[j] = accB[j] = make_float2(0.f, 0.f);
#pragma unroll
          for (int kk = 0; kk < kE / 4; ++kk) {
            const float4 a = ca[kk], b = cbv[kk];
            const float2 a01 = make_float2(a.x, a.y), a23 = make_float2(a.z, a.w);
            const float2 b01 = make_float2(b.x, b.y), b23 = make_float2(b.z, b.w);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int m = 2 * kk + hh;  // bins 2m, 2m+1
              const float4 p01 = bas4[m * (kN / 2) + 2 * q];      // columns 4q, 4q+1
              const float4 p23 = bas4[m * (kN / 2) + 2 * q + 1];  // columns 4q+2, 4q+3
              const float2 cA = hh ? a23 : a01, cB = hh ? b23 : b01;
              accA[0] = __ffma2_rn(cA, make_float2(p01.x, p01.y), accA[0]);
              accA[1] = __ffma2_rn(cA, make_float2(p01.z, p01.w), accA[1]);
              accA[2] = __ffma2_rn(cA, make_float2(p23.x, p23.y), accA[2]);
              accA[3] = __ffma2_rn(cA, make_float2(p23.z, p23.w), accA[3]);
              accB[0] = __ffma2_rn(cB, make_float2(p01.x, p01.y), accB[0]);
              accB[1] = __ffma2_rn(cB, make_float2(p01.z, p01.w), accB[1]);
              accB[2] = __ffma2_rn(cB, make_float2(p23.x, p23.y), accB[2]);
              accB[3] = __ffma2_rn(cB, make_float2(p23.z, p23.w), accB[3]);
            }
          }
          store_window(out, S, (win0 + wa) * kN, q, accA, aligned);
          if (wb < nwin) store_window(out, S, (win0 + wb) * kN, q, accB, aligned);
        }
      }
    }
    __syncwarp();  // the staging entries are rewritten by the next tile
  }
}

template <int WARPS>
void *wptr() {
  return reinterpret_cast<void *>(&k_decode_warp<WARPS>);
}

void *wpick(uint32_t threads) {
  switch (threads) {
    case 128: return wptr<4>();
    case 256: return wptr<8>();
    case 512: return wptr<16>();
    case 1024: return wptr<32>();
    default: return nullptr;
  }
}

}  // namespace

uint32_t warp_tile_windows() { return kT; }

// Shared-memory layout of the warp-tile kernel; returns total bytes, fills wp.
size_t warp_smem_layout(uint32_t threads, const uint32_t *lmax, uint32_t n_domains, WarpParams *wp) {
  size_t o = align16(sizeof(DomW) * (n_domains ? n_domains : 1));
  wp->n_domains = n_domains;
  for (uint32_t d = 0; d < n_domains && d < kWarpMaxDomains; ++d) {
    wp->lut_off[d] = (uint32_t)o;
    o += align16((size_t)2 << lmax[d]);
    wp->tab_off[d] = (uint32_t)o;
    o += align16(3u * kZStride * 4);
  }
  wp->basis_off = (uint32_t)o;
  o += (size_t)(kE / 2) * kN * 8;
  o = align16(o);
  wp->warp_off = (uint32_t)o;
  wp->warp_bytes = (uint32_t)align16((size_t)kPassWords * 8 + 32 + (size_t)kStage * 2 + 2 * (size_t)kStepWin * kRowF * 4);
  return o + (size_t)(threads / 32) * wp->warp_bytes;
}

cudaError_t warp_smem_config(uint32_t threads, size_t smem) {
  void *k = wpick(threads);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return set_dynamic_smem_limit(k, smem);
}

cudaError_t warp_occupancy(uint32_t threads, size_t smem, int *ctas_per_sm) {
  void *k = wpick(threads);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, (int)threads, smem);
}

cudaError_t launch_warp(const DecodeParams &p, const WarpParams &wp, uint32_t threads, uint32_t grid, size_t smem,
                        cudaStream_t stream) {
  if (p.tile_end <= p.tile_begin || grid == 0) return cudaSuccess;
  void *k = wpick(threads);
  if (!k) return cudaErrorInvalidValue;
  DecodeParams pp = p;
  WarpParams ww = wp;
  void *args[] = {&pp, &ww};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
