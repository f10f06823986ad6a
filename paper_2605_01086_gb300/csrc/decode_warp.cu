// Fused decode for the Table 1 shape (N = 32, E = 16) with one warp per tile.
//
// Each warp decodes and transforms its own tile of 64 windows (1024 symbols,
// 2048 samples) with no block-wide barrier in its loop: the SymLen word offsets
// come from a warp scan of symlen, the coefficients go to the warp's own
// shared-memory buffer, and the inverse transform reads them back after a
// __syncwarp.  The decode tables of every domain of the plan stay resident in
// shared memory for the whole kernel (loaded once), so tiles of different
// domains need no reload either.  Warps of the SM interleave decode (shared
// memory / integer work) and transform (FP32 work) of different tiles on their
// own, which the block-tile kernel could only do across CTAs.
//
// Per tile, as in Sec. 4.2: Huffman decode of the tile's words with the
// prefix table (Sec. 3.3), compaction, dequantization by table
// (A_z * unit_z(level)), inverse DCT with window reassembly.  The words of the
// warp's next tile and the tile records two tiles ahead are loaded into
// registers one tile early.
#include "device_util.cuh"

namespace fptc {
namespace {

constexpr int kN = 32;
constexpr int kE = 16;
constexpr int kT = 64;           // windows per tile (about 32 x 4 words at 8-10 symbols per word)
constexpr int kTS = kT * kE;     // symbols per tile
constexpr int kGuard = 64;       // > max skip
constexpr int kZStride = 257;    // zone rows of the dequantization table (bank-conflict padding)

struct WarpTile {
  uint64_t fw;
  uint32_t nw;
  uint32_t skip;
};

__device__ __forceinline__ WarpTile wt_ctx(const SegDev &sg, uint64_t tin, const TileRec &r, const TileRec &rn) {
  WarpTile c;
  c.fw = r.first_word;
  c.skip = r.skip;
  uint64_t lw;
  if (tin + 1 < sg.n_tiles)
    lw = rn.first_word - (rn.skip == 0 ? 1u : 0u);
  else
    lw = sg.word_offset + sg.n_words - 1;
  c.nw = lw >= c.fw ? (uint32_t)(lw - c.fw + 1) : 0u;
  return c;
}

// A lane decodes its WPT consecutive words one after the other (not
// interleaved): the warp then runs for max over lanes of (symbols of the lane's
// words), which varies much less between lanes than the symbols of single
// words do.  Symbol positions q (tile coordinates) start at q0; positions < 0
// go to the guard area; decoding stops at the tile's last symbol.
// n: symbols this lane decodes; nmax: the largest n of the warp (computed by
// the caller with every lane converged).  No warp-synchronous operation in here.
template <int WPT>
__device__ __forceinline__ unsigned wdecode(const uint64_t (&wd)[WPT], const uint32_t (&sl)[WPT], int32_t q0,
                                            uint32_t n, uint32_t nmax, const uint16_t *__restrict__ lut,
                                            uint32_t shift, uint32_t zmask, const float *__restrict__ deq,
                                            float *__restrict__ coef, uint8_t *__restrict__ lev, bool checked,
                                            bool write_lev) {
  uint64_t w[WPT];
  uint32_t r[WPT];
#pragma unroll
  for (int u = 0; u < WPT; ++u) {
    w[u] = wd[u];
    r[u] = sl[u];
  }
  uint32_t hi = (uint32_t)(w[0] >> 32), lo = (uint32_t)w[0], rem = r[0], used = 0;
  int32_t q = q0;
  bool bad = false, over = false;
  for (uint32_t j = 0; j < nmax; ++j) {
    if (j < n) {
      // next word when this one is exhausted (at most WPT - 1 times per lane)
#pragma unroll 1
      for (int guard = 0; rem == 0 && guard < WPT; ++guard) {
        over |= used > 64u;
#pragma unroll
        for (int u = 0; u + 1 < WPT; ++u) {
          w[u] = w[u + 1];
          r[u] = r[u + 1];
        }
        w[WPT - 1] = 0;
        r[WPT - 1] = 0;
        hi = (uint32_t)(w[0] >> 32);
        lo = (uint32_t)w[0];
        rem = r[0];
        used = 0;
      }
      const uint32_t e = lut[hi >> shift];
      const uint32_t len = e >> 8;
      if (checked) bad |= len == 0;
      hi = __funnelshift_l(lo, hi, len);
      lo <<= len;
      used += len;
      const uint32_t sym = e & 0xffu;
      const uint32_t z = (zmask >> (2u * (uint32_t)(q & (kE - 1)))) & 3u;
      coef[q] = deq[z * kZStride + sym];
      if (write_lev) lev[q] = (uint8_t)sym;
      ++q;
      --rem;
    }
  }
  over |= used > 64u;
  return (bad ? kFlagInvalidCode : 0u) | (over ? kFlagBitOverrun : 0u);
}

__device__ __forceinline__ void wstore(float *out, uint64_t S, uint64_t s0, uint32_t q, const float2 (&acc)[4],
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

// Per-domain tables in shared memory: decode table at lut_off (uint16
// entries), then at tab_off the dequantization rows [3][kZStride] (zone 2 row
// zero) followed by the paired basis [8][32] float2.
struct DomSmem {
  uint32_t lut_off;   // bytes
  uint32_t tab_off;   // bytes
  uint32_t shift;     // 32 - lmax
  uint32_t zmask;     // 2 bits per bin: zone of bin k at bits 2k..2k+1
  uint32_t complete;
  uint32_t pad[3];
};

template <int WARPS>
constexpr int warp_min_blocks() {
  return WARPS >= 16 ? 1 : (WARPS >= 8 ? 2 : 4);
}

template <int WARPS, int WPT>
__global__ void __launch_bounds__(WARPS * 32, warp_min_blocks<WARPS>()) k_decode_warp(const DecodeParams p, const WarpParams wp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DomSmem *ds = reinterpret_cast<DomSmem *>(smem_raw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // ---- all domains' tables, once (offsets follow the layout of warp_smem_layout)
  uint32_t off = (uint32_t)align16(sizeof(DomSmem) * (wp.n_domains ? wp.n_domains : 1));
  for (uint32_t d = 0; d < wp.n_domains; ++d) {
    const DomainDev &dm = p.domains[d];
    const uint32_t lut_off = off;
    const uint32_t tab_off = lut_off + (uint32_t)align16((size_t)2 << dm.lmax);
    off = tab_off + (uint32_t)(align16(3u * kZStride * 4) + (size_t)(kE / 2) * kN * 8);
    if (threadIdx.x == 0) {
      DomSmem x;
      x.lut_off = lut_off;
      x.tab_off = tab_off;
      x.shift = 32u - dm.lmax;
      uint32_t zm = 0;
      for (uint32_t k = 0; k < kE; ++k) zm |= (k < dm.B1 ? 0u : (k < dm.B2 ? 1u : 2u)) << (2 * k);
      x.zmask = zm;
      x.complete = dm.complete;
      x.pad[0] = x.pad[1] = x.pad[2] = 0;
      ds[d] = x;
    }
    load_lut<WARPS * 32>(reinterpret_cast<uint16_t *>(smem_raw + lut_off), p.luts + dm.lut_offset, 1u << dm.lmax);
    float a0 = p.scale ? p.scale[d * 3 + 0] : dm.scale[0];
    float a1 = p.scale ? p.scale[d * 3 + 1] : dm.scale[1];
    a0 = a0 > 1e-30f ? a0 : 0.0f;
    a1 = a1 > 1e-30f ? a1 : 0.0f;
    float *deq = reinterpret_cast<float *>(smem_raw + tab_off);
    for (uint32_t i = threadIdx.x; i < 3u * kZStride; i += WARPS * 32) {
      const uint32_t z = i / kZStride, L = i - z * kZStride;
      deq[i] = (L < 256u && z < 2u) ? (z == 0 ? a0 : a1) * dm.unit[z][L] : 0.0f;
    }
    float2 *bp = reinterpret_cast<float2 *>(smem_raw + tab_off + align16(3u * kZStride * 4));
    for (uint32_t i = threadIdx.x; i < (kE / 2) * kN; i += WARPS * 32) {
      const uint32_t m = i / kN, n = i % kN;
      const float *b = p.basis + dm.basis_offset;
      bp[i] = make_float2(__ldg(b + (2 * m) * kN + n), __ldg(b + (2 * m + 1) * kN + n));
    }
  }
  __syncthreads();

  float *const coef = reinterpret_cast<float *>(smem_raw + wp.warp_off + warp * wp.warp_bytes) + kGuard;
  uint8_t *const lev = smem_raw + wp.warp_off + warp * wp.warp_bytes + (kGuard + kTS) * 4 + kGuard;
  const bool want_lev = p.levels != nullptr;
  const uint32_t q = lane & 3u, row = lane >> 2;

  // tiles of this CTA: [t0, t1); warp w takes t0 + w, t0 + w + WARPS, ...
  const uint64_t n_all = p.tile_end - p.tile_begin;
  const uint64_t t0 = p.tile_begin + n_all * blockIdx.x / gridDim.x;
  const uint64_t t1 = p.tile_begin + n_all * (blockIdx.x + 1) / gridDim.x;
  uint64_t g = t0 + warp;
  if (g >= t1) return;
  unsigned err = 0;

  uint32_t s = find_segment(p.segs, p.seg_begin, p.seg_end, g);
  bool cbad = p.seg_bad[s] != 0;
  WarpTile cx{0, 0, 0};
  if (!cbad) {
    const SegDev &sg = p.segs[s];
    const uint64_t tin = g - sg.tile_base;
    TileRec rn{0, 0, 0};
    if (tin + 1 < sg.n_tiles) rn = p.tiles[g + 1];
    cx = wt_ctx(sg, tin, p.tiles[g], rn);
  }
  uint64_t pw[WPT];
  uint32_t psl[WPT];
#pragma unroll
  for (int u = 0; u < WPT; ++u) {
    const uint32_t i = lane * WPT + u;
    const bool in = !cbad && i < cx.nw;
    psl[u] = in ? (uint32_t)__ldg(p.symlen + cx.fw + i) : 0u;
    pw[u] = in ? __ldg(p.words + cx.fw + i) : 0ull;
  }
  // the warp's next tile
  uint64_t g1 = g + WARPS;
  uint32_t s1 = s;
  bool bad1 = true;
  WarpTile c1{0, 0, 0};
  if (g1 < t1) {
    while (g1 >= p.segs[s1].tile_base + p.segs[s1].n_tiles) ++s1;
    bad1 = p.seg_bad[s1] != 0;
    if (!bad1) {
      const SegDev &sg = p.segs[s1];
      const uint64_t tin = g1 - sg.tile_base;
      TileRec rn{0, 0, 0};
      if (tin + 1 < sg.n_tiles) rn = p.tiles[g1 + 1];
      c1 = wt_ctx(sg, tin, p.tiles[g1], rn);
    }
  }

  for (; g < t1; g += WARPS) {
    // ---- loads for later tiles: words of g1, records of g2
    uint64_t nwd[WPT];
    uint32_t nsl[WPT];
#pragma unroll
    for (int u = 0; u < WPT; ++u) {
      const uint32_t i = lane * WPT + u;
      const bool in = g1 < t1 && !bad1 && i < c1.nw;
      nsl[u] = in ? (uint32_t)__ldg(p.symlen + c1.fw + i) : 0u;
      nwd[u] = in ? __ldg(p.words + c1.fw + i) : 0ull;
    }
    const uint64_t g2 = g1 + WARPS;
    uint32_t s2 = s1;
    bool bad2 = true;
    TileRec ra{0, 0, 0}, rb{0, 0, 0};
    if (g2 < t1) {
      while (g2 >= p.segs[s2].tile_base + p.segs[s2].n_tiles) ++s2;
      bad2 = p.seg_bad[s2] != 0;
      if (!bad2) {
        ra = p.tiles[g2];
        if (g2 + 1 - p.segs[s2].tile_base < p.segs[s2].n_tiles) rb = p.tiles[g2 + 1];
      }
    }

    if (!cbad) {
      const SegDev &sg = p.segs[s];
      const uint32_t dom = sg.domain;
      const DomSmem dd = ds[dom];
      const uint64_t tin = g - sg.tile_base;
      const uint64_t win0 = tin * kT;
      const uint64_t left = sg.n_windows - win0;
      const uint32_t nwin = left < (uint64_t)kT ? (uint32_t)left : (uint32_t)kT;
      const int32_t tsyms = (int32_t)(nwin * kE);
      const uint16_t *lut = reinterpret_cast<const uint16_t *>(smem_raw + dd.lut_off);
      const float *deq = reinterpret_cast<const float *>(smem_raw + dd.tab_off);

      // ---- Huffman decode + dequantization into the warp's buffer
      int32_t base = -(int32_t)cx.skip;
      for (uint32_t c0 = 0; c0 < cx.nw; c0 += 32 * WPT) {
        uint64_t wd[WPT];
        uint32_t sl[WPT];
        uint32_t tsum = 0;
#pragma unroll
        for (int u = 0; u < WPT; ++u) {
          if (c0 == 0) {
            wd[u] = pw[u];
            sl[u] = psl[u];
          } else {
            const uint32_t i = c0 + lane * WPT + u;
            const bool in = i < cx.nw;
            sl[u] = in ? (uint32_t)__ldg(p.symlen + cx.fw + i) : 0u;
            wd[u] = in ? __ldg(p.words + cx.fw + i) : 0ull;
          }
          tsum += sl[u];
        }
        uint32_t x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= (uint32_t)o) x += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
        const int32_t q0 = base + (int32_t)(x - tsum);
        const int32_t room = tsyms - q0;
        const uint32_t n = room <= 0 ? 0u : min(tsum, (uint32_t)room);
        const uint32_t nmax = __reduce_max_sync(0xffffffffu, n);  // all 32 lanes are here
        if (n)
          err |= wdecode<WPT>(wd, sl, q0, n, nmax, lut, dd.shift, dd.zmask, deq, coef, lev, dd.complete == 0,
                              want_lev);
        base += (int32_t)total;
        if (base >= tsyms) break;  // uniform over the warp
      }
      if (err) {
        flag_bad(p.status, err, sg.caller_index);
        err = 0;
      }
      __syncwarp();

      if (want_lev) {
        uint8_t *dst = p.levels + sg.level_offset + win0 * kE;
        for (int32_t i = lane; i < tsyms; i += 32) dst[i] = lev[i];
      }
      // ---- inverse transform + reassembly: lane (row, q) does windows
      // row + 16 s and row + 16 s + 8 in step s
      float *out = p.out + sg.out_offset;
      const uint64_t S = sg.n_samples;
      const float4 *bas4 =
          reinterpret_cast<const float4 *>(smem_raw + dd.tab_off + align16(3u * kZStride * 4));  // [m][16]
#pragma unroll 1
      for (int step = 0; step < kT / 16; ++step) {
        const uint32_t wa = row + 16 * step, wb = wa + 8;
        if (wa >= nwin) break;
        const bool two = wb < nwin;
        const float4 *ca = reinterpret_cast<const float4 *>(coef + wa * kE);
        const float4 *cb = reinterpret_cast<const float4 *>(coef + (two ? wb : wa) * kE);
        float2 accA[4], accB[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) accA[j] = accB[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int kk = 0; kk < kE / 4; ++kk) {
          const float4 a = ca[kk], b = cb[kk];
          const float2 a01 = make_float2(a.x, a.y), a23 = make_float2(a.z, a.w);
          const float2 b01 = make_float2(b.x, b.y), b23 = make_float2(b.z, b.w);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int m = 2 * kk + h;
            const float4 p01 = bas4[m * (kN / 2) + 2 * q];
            const float4 p23 = bas4[m * (kN / 2) + 2 * q + 1];
            const float2 cA = h ? a23 : a01, cB = h ? b23 : b01;
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
        wstore(out, S, (win0 + wa) * kN, q, accA, sg.out_aligned);
        if (two) wstore(out, S, (win0 + wb) * kN, q, accB, sg.out_aligned);
      }
      __syncwarp();  // the buffer is rewritten by the next tile
    }

    // ---- rotate
    s = s1;
    cbad = bad1;
    cx = c1;
#pragma unroll
    for (int u = 0; u < WPT; ++u) {
      pw[u] = nwd[u];
      psl[u] = nsl[u];
    }
    g1 = g2;
    s1 = s2;
    bad1 = bad2;
    if (g2 < t1 && !bad2) {
      const SegDev &sgn = p.segs[s2];
      c1 = wt_ctx(sgn, g2 - sgn.tile_base, ra, rb);
    }
  }
}

template <int WARPS, int WPT>
void *wptr() {
  return reinterpret_cast<void *>(&k_decode_warp<WARPS, WPT>);
}

void *wpick(uint32_t threads) {
  switch (threads) {
    case 128: return wptr<4, 4>();
    case 256: return wptr<8, 4>();
    case 512: return wptr<16, 4>();
    default: return nullptr;
  }
}

}  // namespace

uint32_t warp_tile_windows() { return kT; }

// Shared-memory layout of the warp-tile kernel; returns total bytes, fills wp.
size_t warp_smem_layout(uint32_t threads, const uint32_t *lmax, uint32_t n_domains, WarpParams *wp) {
  size_t o = align16(sizeof(DomSmem) * (n_domains ? n_domains : 1));
  wp->n_domains = n_domains;
  for (uint32_t d = 0; d < n_domains && d < kWarpMaxDomains; ++d) {
    wp->lut_off[d] = (uint32_t)o;
    o += align16((size_t)2 << lmax[d]);
    wp->tab_off[d] = (uint32_t)o;
    o += align16(3u * kZStride * 4) + (size_t)(kE / 2) * kN * 8;
  }
  o = align16(o);
  wp->warp_off = (uint32_t)o;
  wp->warp_bytes = (uint32_t)align16((size_t)(kGuard + kTS) * 4 + kGuard + kTS);
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
