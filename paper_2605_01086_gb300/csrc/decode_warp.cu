// Fused decode for the Table 1 shape (N = 32, E = 16) with one warp per tile.
//
// Each warp owns a contiguous range of tiles of 128 windows (2048 symbols, 4096
// samples) and runs Sec. 4.2 on each with no block-wide barrier:
//  1. SymLen decode.  A pass gives every lane two consecutive words; a warp
//     scan of their symbol counts places each word's codewords (compaction,
//     Sec. 4.2.1).  A lane decodes a word with one decode-table lookup per
//     codeword and stores the codeword's level as one byte at its tile
//     position (two per 16-bit store).  Nothing else happens per
//     codeword: the dequantization waits for step 2, where the bin of every
//     value is known at compile time.  The 64-bit word is shifted through
//     hi:lo with a marker bit under it, so a word whose codewords need more
//     than 64 bits shows as an empty buffer at the end (no per-codeword count).
//  2. Dequantization and inverse DCT, one window per lane.  The lane reads its
//     window's 16 levels, turns each into A_z * unit_z(level) (one table read;
//     the bin, hence the zone row, is fixed per register), and evaluates the
//     inverse of Eq. 1 by the even/odd split of the DCT-III:
//     x[n] = E[n] + O[n], x[31-n] = E[n] - O[n] with O the odd bins and E the
//     even bins, itself split the same way twice (E[15-n] = EE[n] - EO[n],
//     EE[7-n] = EEE[n] - EEO[n]); 229 FP32 operations per window with the
//     cosines as compile-time constants, so neither a basis nor coefficients
//     pass through shared memory.
//  3. Output.  Where the segment's output starts on a 128-byte boundary and
//     all 32 windows of a step are whole, the lanes write their windows into
//     the warp's shared staging tile in the 128-byte swizzled layout (chunk c
//     of row r at c ^ (r & 7): conflict-free) and one lane stores the tile
//     with a TMA tensor store (the output viewed as rows of 32 floats), so the
//     output never passes through the L1 load/store pipe.  Other windows use
//     32-byte (or 16-byte, or scalar) streaming stores.
//  The warp locates the first tile of its range from the index's chunk
//  offsets; tile g+1 starts at the word where tile g's decode ended, and its
//  first words are loaded then (hidden by tile g's transform); the words of a
//  tile's next decode pass load while the current pass decodes.
// The decode tables, dequantization rows and basis of every domain stay in
// shared memory for the whole kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "warp_tile.cuh"

namespace fptc {
namespace {

using namespace wt;

// ---- compile-time cosines of the inverse transform (N = 32, E = 16) ----------
// cos(pi num / den) in double: Taylor series on [0, pi/2] after the reflections
// cos(2 pi - a) = cos(a) and cos(pi - a) = -cos(a); rounded to float.
__host__ __device__ constexpr double cos_taylor(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int i = 1; i < 24; ++i) {
    term *= -x2 / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr float cospi_frac(int num, int den) {
  int r = num % (2 * den);
  if (r > den) r = 2 * den - r;
  const double pi = 3.14159265358979323846;
  return 2 * r <= den ? (float)cos_taylor(pi * r / den) : (float)-cos_taylor(pi * (den - r) / den);
}
// B[k][n] = cos(pi (2n+1) k / 64) grouped by the even/odd recursion:
//   eee[n]    = B[8][n]                       n < 4
//   eeo[n][j] = B[4(2j+1)][n]                 n < 4, j < 2   (bins 4, 12)
//   eo[n][j]  = B[2(2j+1)][n]                 n < 8, j < 4   (bins 2, 6, 10, 14)
//   o[n][j]   = B[2j+1][n]                    n < 16, j < 8  (odd bins)
struct IdctK {
  float eee[4];
  float eeo[4][2];
  float eo[8][4];
  float o[16][8];
};
__host__ __device__ constexpr IdctK make_idct_k() {
  IdctK K{};
  for (int n = 0; n < 4; ++n) K.eee[n] = cospi_frac(2 * n + 1, 8);
  for (int n = 0; n < 4; ++n)
    for (int j = 0; j < 2; ++j) K.eeo[n][j] = cospi_frac((2 * n + 1) * (2 * j + 1), 16);
  for (int n = 0; n < 8; ++n)
    for (int j = 0; j < 4; ++j) K.eo[n][j] = cospi_frac((2 * n + 1) * (2 * j + 1), 32);
  for (int n = 0; n < 16; ++n)
    for (int j = 0; j < 8; ++j) K.o[n][j] = cospi_frac((2 * n + 1) * (2 * j + 1), 64);
  return K;
}

// x[0..31] of one window from its 16 coefficients (inverse of Eq. 1, B[0][n] = 1/2);
// emits the samples as four blocks of 8 through put(block, v[8]).
template <class Put>
__device__ __forceinline__ void idct32(const float (&c)[16], Put put) {
  constexpr IdctK K = make_idct_k();
  const float h0 = 0.5f * c[0];
  float ee[8], eo[8];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const float eee = fmaf(c[8], K.eee[n], h0);
    const float eeo = fmaf(c[12], K.eeo[n][1], c[4] * K.eeo[n][0]);
    ee[n] = eee + eeo;
    ee[7 - n] = eee - eeo;
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    float a = c[2] * K.eo[n][0];
    a = fmaf(c[6], K.eo[n][1], a);
    a = fmaf(c[10], K.eo[n][2], a);
    eo[n] = fmaf(c[14], K.eo[n][3], a);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float lo[8], hi[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int n = 8 * j + i;
      const float e = n < 8 ? ee[n] + eo[n] : ee[15 - n] - eo[15 - n];
      float o = c[1] * K.o[n][0];
#pragma unroll
      for (int t = 1; t < 8; ++t) o = fmaf(c[2 * t + 1], K.o[n][t], o);
      lo[i] = e + o;       // x[n]
      hi[7 - i] = e - o;   // x[31 - n]
    }
    put(j, lo);
    put(3 - j, hi);
  }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, WARPS > 16 ? 1 : 32 / WARPS) k_decode_warp(
    const DecodeParams p, const WarpParams wp, const __grid_constant__ CUtensorMap out_map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DomW *const dw = reinterpret_cast<const DomW *>(smem_raw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  load_domain_tables<WARPS * 32>(p, wp.n_domains, smem_raw);
  __syncthreads();

  unsigned char *const wbase = smem_raw + wp.warp_off + warp * kMiscBytes;
  uint64_t *const wbuf = reinterpret_cast<uint64_t *>(wbase);                       // first-pass words
  uint8_t *const stage = wbase + kStageOff;                           // tile position 0
  // output staging tile: 1024-byte aligned (the period of the 128-byte swizzle)
  const uintptr_t tiles0 = (reinterpret_cast<uintptr_t>(smem_raw + wp.warp_off + WARPS * kMiscBytes) + 1023) &
                           ~uintptr_t(1023);
  unsigned char *const otile = reinterpret_cast<unsigned char *>(tiles0) + warp * kOutTile;
  const bool want_lev = p.levels != nullptr;
  bool tma_pending = false;

  // ---- this warp's tiles: an even split of the launch's tile range over all warps
  uint64_t tw0, tw1;
  unit_tiles(p, (uint64_t)blockIdx.x * WARPS + warp, (uint64_t)gridDim.x * WARPS, tw0, tw1);
  if (tw0 >= tw1) return;

  // prologue: where tile tw0 starts, then its first words
  Ctx nxt = first_ctx(p, find_segment(p.segs, p.seg_begin, p.seg_end, tw0), tw0, lane);
  uint32_t pn = fetch_pass0(p, nxt, lane, wbuf);

  for (uint64_t g = tw0; g < tw1; ++g) {
    // ---- tile g: its first words have been requested
    cp_async_wait_all();
    __syncwarp();
    const Ctx cur = nxt;
    uint64_t w[kWPL];
    uint32_t n[kWPL];
#pragma unroll
    for (int u = 0; u < kWPL; ++u) {
      w[u] = wbuf[kWPL * lane + u];
      n[u] = (pn >> (8 * u)) & 0xffu;
    }
    __syncwarp();
    const uint64_t g1 = g + 1;

    const SegDev &sg = p.segs[cur.seg];
    const DomW dd = dw[sg.domain];
    const uint64_t win0 = (g - sg.tile_base) * kT;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = left < (uint64_t)kT ? (uint32_t)left : (uint32_t)kT;

    // ---- 1. SymLen decode into the level bytes
    TileEnd te{0u, 0u, 0u};
    if (cur.ok) {
      te = decode_tile(p, cur, nwin * kE, dd, smem_raw, stage, lane, w, n);
      if (te.bad && lane == 0) flag_bad(p.status, te.bad, sg.caller_index);
    }

    // ---- first words of tile g + 1 (in flight during the transform)
    if (g1 < tw1) {
      nxt = next_ctx(p, g, cur.seg, cur, te);
      pn = fetch_pass0(p, nxt, lane, wbuf);
    }
    __syncwarp();

    // ---- 2./3. dequantization + inverse transform + reassembly, one window per lane
    if (cur.ok) {
      const float *deq = reinterpret_cast<const float *>(smem_raw + dd.deq_off);
      float *const out = p.out + sg.out_offset;
      const uint64_t S = sg.n_samples;
      const uint32_t aligned = sg.out_aligned;
      const bool vec32 = (aligned & 2u) && (reinterpret_cast<uintptr_t>(p.out) & 31u) == 0;
      const bool tma_seg = wp.out_tma && (aligned & 4u);
      uint8_t *const lev = want_lev ? p.levels + sg.level_offset + win0 * kE : nullptr;
#pragma unroll 1
      for (uint32_t w0 = 0; w0 < nwin; w0 += kStepWin) {
        const uint32_t wi = w0 + lane;
        // all 32 windows of the step whole and inside the segment: one TMA store
        const bool tma_step = tma_seg && w0 + kStepWin <= nwin && (win0 + w0 + kStepWin) * kN <= S;
        if (tma_pending) {
          if (lane == 0) tma_wait_read();  // the previous step has left the staging tile
          __syncwarp();
          tma_pending = false;
        }
        // row `lane` of the staging tile, 16-byte chunk c at c ^ (lane & 7)
        unsigned char *const row = otile + lane * (kN * 4);
        const uint32_t sx = lane & 7u;
        if (wi < nwin) {
          const uint4 sv = *reinterpret_cast<const uint4 *>(stage + wi * kE);
          float c[16];
          window_coefs(sv, deq, dd.zmask, c);
          if (want_lev) put_levels(lev + wi * kE, sv);
          idct32(c, [&](int b, const float(&v)[8]) {
            *reinterpret_cast<float4 *>(row + (((2 * b) ^ sx) << 4)) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4 *>(row + (((2 * b + 1) ^ sx) << 4)) = make_float4(v[4], v[5], v[6], v[7]);
          });
        }
        if (tma_step) {
          fence_async_shared();
          __syncwarp();
          if (lane == 0) tma_store_rows(&out_map, otile, (int32_t)((sg.out_offset >> 5) + win0 + w0));
          tma_pending = true;
        } else if (wi < nwin) {  // each lane stores its own row
          const uint64_t s0 = (win0 + wi) * kN;
          store_row(row, sx, out + s0, s0 + kN <= S ? kN : (uint32_t)(S - s0), vec32, aligned & 1u);
        }
      }
    }
    __syncwarp();  // the level bytes are rewritten by the next tile
  }
  if (tma_pending && lane == 0) tma_wait_all();
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
    case 768: return wptr<24>();
    case 896: return wptr<28>();
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
    o += kDeqBytes;
  }
  o = align16(o);
  wp->warp_off = (uint32_t)o;
  wp->warp_bytes = (uint32_t)kMiscBytes;
  wp->out_tma = 0;
  const size_t warps = threads / 32;
  return o + warps * kMiscBytes + 1023 + warps * kOutTile;  // + alignment of the staging tiles
}

bool encode_out_map(CUtensorMap *map, float *out, uint64_t extent) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  const uint64_t rows = extent / kN;
  if (!encode || !out || (reinterpret_cast<uintptr_t>(out) & 15u) || rows == 0 || rows > 0x7FFFFFFFull) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kN, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kN * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kN, (cuuint32_t)kStepWin};
  const cuuint32_t estride[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, out, dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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

cudaError_t launch_warp(const DecodeParams &p, const WarpParams &wp, const CUtensorMap &out_map, uint32_t threads,
                        uint32_t grid, size_t smem, cudaStream_t stream) {
  if (p.tile_end <= p.tile_begin || grid == 0) return cudaSuccess;
  void *k = wpick(threads);
  if (!k) return cudaErrorInvalidValue;
  DecodeParams pp = p;
  WarpParams ww = wp;
  CUtensorMap mm = out_map;
  void *args[] = {&pp, &ww, &mm};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
