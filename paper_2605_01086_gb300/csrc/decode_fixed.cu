// Fused decode for the Table 1 shape (N = 32, E = 16), software-pipelined.
//
// Same work per tile as the generic kernel (Sec. 4.2: SymLen Huffman decode with
// the decode table in shared memory, compaction by a block scan of symlen,
// dequantization, inverse DCT, window reassembly), organised for GB300:
//  - each thread owns WPT consecutive words of a tile and decodes them
//    interleaved (WPT independent dependency chains per thread); the 64-bit
//    bit buffer is kept as two 32-bit halves and advanced with a funnel shift;
//  - the words/symlen of tile g+1 and the tile records of tile g+2 are loaded
//    into registers at the start of tile g, so the two dependent HBM round
//    trips of a tile (tile start, then its words) overlap a whole tile of work;
//  - dequantization is one shared-memory lookup in a per-bin table
//    deq[k][level] = A_zone(k) * unit_zone(k)(level) (zone 2 rows are zero);
//    symbols that belong to the previous tile land in a guard area in front of
//    the coefficient buffer, so the decode loop has no bounds test;
//  - coefficient buffers alternate between tiles, so one barrier per tile
//    separates decoding from the inverse transform;
//  - the inverse transform pairs even and odd bins in FFMA2 (two FP32 FMAs per
//    instruction): acc = sum_m (c[2m], c[2m+1]) * (B[2m][n], B[2m+1][n]); by the
//    mirror symmetry B[k][N-1-n] = (-1)^k B[k][n], x[n] = acc.x + acc.y and
//    x[N-1-n] = acc.x - acc.y, i.e. 8 multiply-adds per sample; the paired
//    basis comes from shared memory and serves two windows per step; stores
//    are 16-byte streaming stores.
#include "device_util.cuh"

namespace fptc {
namespace {

constexpr int kN = 32;
constexpr int kE = 16;
constexpr int kQ = kN / 8;      // threads per window (4 samples + their 4 mirrors each)
constexpr int kGuard = 64;      // > max skip (a word holds at most 64 symbols)
// Row stride of the per-bin dequantization table.  257 = 256 + 1 puts the same
// level of different bins in different shared-memory banks (the zero level 128
// dominates every bin, and with a stride of 256 all bins would share bank 0).
constexpr int kDeqStride = 257;

struct FSmem {
  uint16_t *lut;
  float *deq;      // [16][kDeqStride]
  float2 *basis;   // [8][32]: (B[2m][n], B[2m+1][n])
  float *coef[2];  // kGuard + coef_cap each; position 0 at coef + kGuard
  uint8_t *lev[2]; // kGuard + coef_cap each
  uint32_t *scan;
};

__device__ __forceinline__ FSmem fcarve(unsigned char *base, uint32_t lut_cap, uint32_t coef_cap) {
  FSmem s;
  size_t o = 0;
  s.lut = reinterpret_cast<uint16_t *>(base + o);
  o += align16((size_t)lut_cap * 2);
  s.deq = reinterpret_cast<float *>(base + o);
  o += align16((size_t)kE * kDeqStride * 4);
  s.basis = reinterpret_cast<float2 *>(base + o);
  o += (size_t)kE * kN * 4;
  for (int b = 0; b < 2; ++b) {
    s.coef[b] = reinterpret_cast<float *>(base + o);
    o += align16(((size_t)kGuard + coef_cap) * 4);
  }
  for (int b = 0; b < 2; ++b) {
    s.lev[b] = base + o;
    o += align16((size_t)kGuard + coef_cap);
  }
  s.scan = reinterpret_cast<uint32_t *>(base + o);
  return s;
}

// Where a tile's words are: first word, word count, symbols of the first word
// that belong to the previous tile.
struct TileCtx {
  uint64_t fw;
  uint32_t nw;
  uint32_t skip;
};

__device__ __forceinline__ TileCtx tile_ctx(const SegDev &sg, uint64_t tin, const TileRec &r, const TileRec &rn) {
  TileCtx c;
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

// Decode WPT consecutive words interleaved.  Symbol positions q (tile
// coordinates) start at q0; positions < 0 go to the guard area; decoding of a
// word stops at the tile's last symbol.
template <int WPT, bool CHECKED, bool WRITE_LEV>
__device__ __forceinline__ unsigned decode_words(const uint64_t (&wd)[WPT], const uint32_t (&sl)[WPT], int32_t q0,
                                                 int32_t tsyms, const uint16_t *__restrict__ lut, uint32_t shift,
                                                 const float *__restrict__ deq, float *__restrict__ coef,
                                                 uint8_t *__restrict__ lev) {
  uint32_t hi[WPT], lo[WPT];
  int32_t q[WPT];
  uint32_t cnt[WPT], used[WPT];
  uint32_t maxc = 0;
  int32_t qq = q0;
#pragma unroll
  for (int u = 0; u < WPT; ++u) {
    hi[u] = (uint32_t)(wd[u] >> 32);
    lo[u] = (uint32_t)wd[u];
    q[u] = qq;
    const int32_t room = tsyms - qq;
    cnt[u] = room <= 0 ? 0u : min(sl[u], (uint32_t)room);
    qq += (int32_t)sl[u];
    used[u] = 0;
    maxc = max(maxc, cnt[u]);
  }
  bool bad = false;
  for (uint32_t j = 0; j < maxc; ++j) {
#pragma unroll
    for (int u = 0; u < WPT; ++u) {
      if (j < cnt[u]) {
        const uint32_t e = lut[hi[u] >> shift];
        const uint32_t len = e >> 8;  // <= 16
        if (CHECKED) bad |= len == 0;
        hi[u] = __funnelshift_l(lo[u], hi[u], len);
        lo[u] <<= len;
        used[u] += len;
        const uint32_t sym = e & 0xffu;
        coef[q[u]] = deq[(uint32_t)(q[u] & (kE - 1)) * kDeqStride + sym];
        if (WRITE_LEV) lev[q[u]] = (uint8_t)sym;
        ++q[u];
      }
    }
  }
  unsigned err = bad ? kFlagInvalidCode : 0u;
#pragma unroll
  for (int u = 0; u < WPT; ++u)
    if (used[u] > 64u) err |= kFlagBitOverrun;
  return err;
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

template <int THREADS>
constexpr int fixed_min_blocks() {
  return THREADS >= 512 ? 2 : (THREADS >= 256 ? 3 : 4);
}

template <int THREADS, int WPT>
__global__ void __launch_bounds__(THREADS, fixed_min_blocks<THREADS>()) k_decode_fixed(const DecodeParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FSmem sm = fcarve(smem_raw, p.lut_cap, p.coef_cap);
  constexpr uint32_t kPass = THREADS * WPT;  // words decoded per block pass

  const uint64_t n_all = p.tile_end - p.tile_begin;
  const uint64_t t0 = p.tile_begin + n_all * blockIdx.x / gridDim.x;
  const uint64_t t1 = p.tile_begin + n_all * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;

  const bool want_lev = p.levels != nullptr;
  const uint32_t q = threadIdx.x % kQ;
  uint32_t cur_dom = 0xFFFFFFFFu;
  bool complete = true;
  uint32_t shift = 20;
  unsigned err = 0;

  // ---- prologue: contexts of tiles t0 and t0+1, words of t0
  uint32_t s = find_segment(p.segs, p.seg_begin, p.seg_end, t0);
  TileCtx cx{0, 0, 0};
  bool cbad = p.seg_bad[s] != 0;
  if (!cbad) {
    const SegDev &sg = p.segs[s];
    const uint64_t tin = t0 - sg.tile_base;
    TileRec rn{0, 0, 0};
    if (tin + 1 < sg.n_tiles) rn = p.tiles[t0 + 1];
    cx = tile_ctx(sg, tin, p.tiles[t0], rn);
  }
  uint64_t pw[WPT];
  uint32_t psl[WPT];
#pragma unroll
  for (int u = 0; u < WPT; ++u) {
    const uint32_t i = threadIdx.x * WPT + u;
    const bool in = !cbad && i < cx.nw;
    psl[u] = in ? (uint32_t)__ldg(p.symlen + cx.fw + i) : 0u;
    pw[u] = in ? __ldg(p.words + cx.fw + i) : 0ull;
  }
  uint32_t s1 = s;
  bool bad1 = true;
  TileCtx c1{0, 0, 0};
  if (t0 + 1 < t1) {
    while (t0 + 1 >= p.segs[s1].tile_base + p.segs[s1].n_tiles) ++s1;
    bad1 = p.seg_bad[s1] != 0;
    if (!bad1) {
      const SegDev &sg = p.segs[s1];
      const uint64_t tin = t0 + 1 - sg.tile_base;
      TileRec rn{0, 0, 0};
      if (tin + 1 < sg.n_tiles) rn = p.tiles[t0 + 2];
      c1 = tile_ctx(sg, tin, p.tiles[t0 + 1], rn);
    }
  }

  uint32_t buf = 0;
  for (uint64_t g = t0; g < t1; ++g, buf ^= 1u) {
    // ---- issue the loads of tile g+1's words and of tile g+2's records; they
    // are consumed one iteration later
    uint64_t nwd[WPT];
    uint32_t nsl[WPT];
#pragma unroll
    for (int u = 0; u < WPT; ++u) {
      const uint32_t i = threadIdx.x * WPT + u;
      const bool in = g + 1 < t1 && !bad1 && i < c1.nw;
      nsl[u] = in ? (uint32_t)__ldg(p.symlen + c1.fw + i) : 0u;
      nwd[u] = in ? __ldg(p.words + c1.fw + i) : 0ull;
    }
    const uint64_t g2 = g + 2;
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

    const SegDev &sg = p.segs[s];
    const uint32_t dom = sg.domain;
    const DomainDev &dm = p.domains[dom];
    const uint64_t tin = g - sg.tile_base;
    const uint32_t T = dm.tile_windows;
    const uint64_t win0 = tin * T;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = left < T ? (uint32_t)left : T;
    const int32_t tsyms = (int32_t)(nwin * kE);
    // select, not index: a dynamic index into sm's arrays would put sm in local memory
    float *const coefg = (buf ? sm.coef[1] : sm.coef[0]) + kGuard;
    uint8_t *const levg = (buf ? sm.lev[1] : sm.lev[0]) + kGuard;

    if (!cbad) {
      if (dom != cur_dom) {
        __syncthreads();
        load_lut<THREADS>(sm.lut, p.luts + dm.lut_offset, 1u << dm.lmax);
        float a0 = p.scale ? p.scale[dom * 3 + 0] : dm.scale[0];
        float a1 = p.scale ? p.scale[dom * 3 + 1] : dm.scale[1];
        a0 = a0 > 1e-30f ? a0 : 0.0f;
        a1 = a1 > 1e-30f ? a1 : 0.0f;
        for (uint32_t i = threadIdx.x; i < kE * 256u; i += THREADS) {
          const uint32_t k = i >> 8, L = i & 255u;
          const uint32_t z = k < dm.B1 ? 0u : (k < dm.B2 ? 1u : 2u);
          sm.deq[k * kDeqStride + L] = z == 0 ? a0 * dm.unit[0][L] : (z == 1 ? a1 * dm.unit[1][L] : 0.0f);
        }
        for (uint32_t i = threadIdx.x; i < (kE / 2) * kN; i += THREADS) {
          const uint32_t m = i / kN, n = i % kN;
          const float *b = p.basis + dm.basis_offset;
          sm.basis[i] = make_float2(__ldg(b + (2 * m) * kN + n), __ldg(b + (2 * m + 1) * kN + n));
        }
        cur_dom = dom;
        complete = dm.complete != 0;
        shift = 32u - dm.lmax;
        __syncthreads();
      }

      // ---- Huffman decode + dequantization into shared memory
      int32_t base = -(int32_t)cx.skip;
      for (uint32_t c0 = 0; c0 < cx.nw; c0 += kPass) {
        uint64_t wd[WPT];
        uint32_t sl[WPT];
        uint32_t tsum = 0;
#pragma unroll
        for (int u = 0; u < WPT; ++u) {
          if (c0 == 0) {
            wd[u] = pw[u];
            sl[u] = psl[u];
          } else {
            const uint32_t i = c0 + threadIdx.x * WPT + u;
            const bool in = i < cx.nw;
            sl[u] = in ? (uint32_t)__ldg(p.symlen + cx.fw + i) : 0u;
            wd[u] = in ? __ldg(p.words + cx.fw + i) : 0ull;
          }
          tsum += sl[u];
        }
        uint32_t total;
        const uint32_t ex = block_exclusive_scan<THREADS>(tsum, sm.scan, &total);
        if (tsum) {
          const int32_t q0 = base + (int32_t)ex;
          if (complete) {
            if (want_lev)
              err |= decode_words<WPT, false, true>(wd, sl, q0, tsyms, sm.lut, shift, sm.deq, coefg, levg);
            else
              err |= decode_words<WPT, false, false>(wd, sl, q0, tsyms, sm.lut, shift, sm.deq, coefg, levg);
          } else {
            if (want_lev)
              err |= decode_words<WPT, true, true>(wd, sl, q0, tsyms, sm.lut, shift, sm.deq, coefg, levg);
            else
              err |= decode_words<WPT, true, false>(wd, sl, q0, tsyms, sm.lut, shift, sm.deq, coefg, levg);
          }
        }
        base += (int32_t)total;
        if (base >= tsyms) break;  // uniform
      }
      if (err) {
        flag_bad(p.status, err, sg.caller_index);
        err = 0;
      }
    }
    // The coefficient buffers alternate between tiles: this barrier separates
    // the decode of tile g from its transform, and (with the barriers of the
    // next tile's scan) the transform of tile g from the decode of tile g+2.
    __syncthreads();

    if (!cbad) {
      if (want_lev) {
        uint8_t *dst = p.levels + sg.level_offset + win0 * kE;
        for (int32_t i = threadIdx.x; i < tsyms; i += THREADS) dst[i] = levg[i];
      }
      // ---- inverse transform + window reassembly, two windows per step
      float *out = p.out + sg.out_offset;
      const uint64_t S = sg.n_samples;
      const uint32_t aligned = sg.out_aligned;
      const float4 *bas4 = reinterpret_cast<const float4 *>(sm.basis);  // [m][16] float4 = 2 columns
      constexpr uint32_t kRows = THREADS / kQ;
      for (uint32_t wa = threadIdx.x / kQ; wa < nwin; wa += 2 * kRows) {
        const uint32_t wb = wa + kRows;
        const bool two = wb < nwin;
        const float4 *ca = reinterpret_cast<const float4 *>(coefg + wa * kE);
        const float4 *cb = reinterpret_cast<const float4 *>(coefg + (two ? wb : wa) * kE);
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
            const int m = 2 * kk + h;  // bins 2m, 2m+1
            const float4 p01 = bas4[m * (kN / 2) + 2 * q];      // columns 4q, 4q+1
            const float4 p23 = bas4[m * (kN / 2) + 2 * q + 1];  // columns 4q+2, 4q+3
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
        store_window(out, S, (win0 + wa) * kN, q, accA, aligned);
        if (two) store_window(out, S, (win0 + wb) * kN, q, accB, aligned);
      }
    }

    // ---- rotate the pipeline: g+1 becomes current, g+2 becomes next
    s = s1;
    cbad = bad1;
    cx = c1;
#pragma unroll
    for (int u = 0; u < WPT; ++u) {
      pw[u] = nwd[u];
      psl[u] = nsl[u];
    }
    s1 = s2;
    bad1 = bad2;
    if (g2 < t1 && !bad2) {
      const SegDev &sgn = p.segs[s2];
      c1 = tile_ctx(sgn, g2 - sgn.tile_base, ra, rb);
    }
  }
}

template <int THREADS, int WPT>
void *fixed_ptr() {
  return reinterpret_cast<void *>(&k_decode_fixed<THREADS, WPT>);
}

void *fpick(uint32_t threads) {
  switch (threads) {
    case 128: return fixed_ptr<128, 4>();
    case 256: return fixed_ptr<256, 2>();
    case 512: return fixed_ptr<512, 1>();
    default: return nullptr;
  }
}

}  // namespace

size_t fixed_smem_bytes(uint32_t threads, uint32_t lut_cap, uint32_t coef_cap) {
  return align16((size_t)lut_cap * 2) + align16((size_t)kE * kDeqStride * 4) + (size_t)kE * kN * 4 +
         2 * align16(((size_t)kGuard + coef_cap) * 4) + 2 * align16((size_t)kGuard + coef_cap) +
         (size_t)(threads / 32) * 4;
}

cudaError_t fixed_smem_config(uint32_t threads, size_t smem) {
  void *k = fpick(threads);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return set_dynamic_smem_limit(k, smem);
}

cudaError_t fixed_occupancy(uint32_t threads, size_t smem, int *ctas_per_sm) {
  void *k = fpick(threads);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, (int)threads, smem);
}

cudaError_t launch_fixed(const DecodeParams &p, uint32_t threads, uint32_t grid, size_t smem, cudaStream_t stream) {
  if (p.tile_end <= p.tile_begin || grid == 0) return cudaSuccess;
  void *k = fpick(threads);
  if (!k) return cudaErrorInvalidValue;
  DecodeParams pp = p;
  void *args[] = {&pp};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
