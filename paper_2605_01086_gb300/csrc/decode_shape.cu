// Fused decode for window shapes other than the Table 1 default: every domain of
// the plan has a window size N in [4, 128] and any kept-bin count E <= N,
// domains of different N in one batch (Table 1 gives the ranges; Fig. 14
// measures how the throughput moves with them).  The transform is compiled per
// power-of-two N and chosen per tile from the tile's domain (a warp-uniform
// switch); other N take a run-time-N version (shape_transform_any).
//
// The SymLen decode, tile chaining, level staging and TMA output path are those
// of the warp-tile kernel (warp_tile.cuh), with tiles of T windows per domain
// (about 2048 symbols, a whole number of output steps).  The transform differs:
// a step is 1024 consecutive samples of a tile (R = 1024 / N windows, the 32 x 32
// staging tile), and every lane computes 32 of them as 16 pairs
// (n, N - 1 - n) of one window (N >= 32: N / 32 lanes per window, lane q of a
// window taking n in [16 q, 16 q + 16)) or of 32 / N windows (N < 32).  The
// inverse of Eq. 1 is evaluated by the mirror symmetry of its basis,
// B[k][N - 1 - n] = (-1)^k B[k][n]:
//     x[n] = Ev[n] + Od[n],  x[N - 1 - n] = Ev[n] - Od[n],
// with Ev / Od the sums over even / odd bins k < min(E, B2) (bins from B2 on
// reconstruct to zero), E / 2 FMAs per sample.  Each bin's coefficient is one
// dequantization-table read (shared by the lanes of a window); the basis
// values B[k][n] for n < N / 2 sit in shared memory, padded so that the lanes
// of a warp read them as broadcasts without bank conflicts.
#include <cuda.h>

#include "warp_tile.cuh"

namespace fptc {
namespace {

using namespace wt;

// Per-domain view of the shared tables of the shape kernel.
struct DomS {
  uint32_t lut_off;    // bytes from the start of shared memory (entries len | level << 8)
  uint32_t deq_off;    // bytes: zone rows [3][kZStride] floats
  uint32_t basis_off;  // bytes: [E][brow] floats
  uint32_t shift;      // 32 - lmax
  uint32_t complete;
  uint32_t E, B1, kz;  // kz = min(E, B2)
  uint32_t T;          // windows per tile
  uint32_t N;
  uint32_t pad[2];
};

template <int N>
struct ShapeK {
  static constexpr int L = N >= 32 ? N / 32 : 1;   // lanes per window
  static constexpr int M = N >= 32 ? 1 : 32 / N;   // windows per lane
  static constexpr int P = N >= 32 ? 16 : N / 2;   // sample pairs per window and lane
  static constexpr int R = 1024 / N;               // windows per step
  // basis floats per bin: N >= 32, 16 values (+ 4 pad) per lane group q; N < 32, the N / 2 values
  static constexpr int BROW = N >= 32 ? L * 20 : (P + 3) / 4 * 4;
  static_assert(M * P == 16, "16 pairs per lane");
};

__host__ __device__ constexpr bool shape_pow2(uint32_t N) { return (N & (N - 1)) == 0; }
// Other N: the ceil(N / 2) sample pairs of a window in groups of 16, one lane per group.
__host__ __device__ constexpr uint32_t shape_any_pairs(uint32_t N) { return (N + 1) / 2; }
__host__ __device__ constexpr uint32_t shape_any_lanes(uint32_t N) { return (shape_any_pairs(N) + 15) / 16; }
// Windows per output step for other N: one lane group each, at most 1024 samples.
__host__ __device__ constexpr uint32_t shape_any_step(uint32_t N) {
  return 32 / shape_any_lanes(N) < 1024 / N ? 32 / shape_any_lanes(N) : 1024 / N;
}

__host__ __device__ constexpr uint32_t shape_brow(uint32_t N) {
  return !shape_pow2(N) ? shape_any_lanes(N) * 20 : N >= 32 ? N / 32 * 20 : (N / 2 + 3) / 4 * 4;
}

// Windows per tile for a domain of the shape kernel: whole steps of 1024
// samples, at most 2048 symbols (the level staging buffer) and at most 8 steps
// (8192 samples: the dL/dx tile of the block adjoint fits shared memory).
__host__ __device__ constexpr uint32_t shape_tile_windows(uint32_t N, uint32_t E) {
  const uint32_t r = shape_pow2(N) ? 1024 / N : shape_any_step(N);
  uint32_t t = (uint32_t)kTS / E / r * r;
  if (t > 8 * r) t = 8 * r;
  return t ? t : r;
}

// Tables of every domain into shared memory from byte 0 (the layout of
// shape_smem_layout).  Returns the end offset.  Contains no barrier.
template <int THREADS>
__device__ __forceinline__ uint32_t load_shape_tables(const DecodeParams &p, uint32_t n_domains, unsigned char *smem) {
  DomS *const ds = reinterpret_cast<DomS *>(smem);
  uint32_t off = (uint32_t)align16(sizeof(DomS) * (n_domains ? n_domains : 1));
  for (uint32_t d = 0; d < n_domains; ++d) {
    const DomainDev &dm = p.domains[d];
    const uint32_t N = dm.N, brow = shape_brow(N), half = N / 2;
    const uint32_t lut_off = off;
    const uint32_t deq_off = lut_off + (uint32_t)align16((size_t)2 << dm.lmax);
    const uint32_t basis_off = deq_off + (uint32_t)align16(3u * kZStride * 4);
    off = basis_off + (uint32_t)align16((size_t)dm.E * brow * 4);
    if (threadIdx.x == 0) {
      DomS x;
      x.lut_off = lut_off;
      x.deq_off = deq_off;
      x.basis_off = basis_off;
      x.shift = 32u - dm.lmax;
      x.complete = dm.complete;
      x.E = dm.E;
      x.B1 = dm.B1;
      x.kz = dm.B2 < dm.E ? dm.B2 : dm.E;
      x.T = dm.tile_windows;
      x.N = N;
      x.pad[0] = x.pad[1] = 0;
      ds[d] = x;
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
    // the half basis B[k][n], n < ceil(N / 2): rows of brow floats, in groups of 16 (+ 4
    // pad) for N >= 32 and for N not a power of two
    float *bas = reinterpret_cast<float *>(smem + basis_off);
    const float *g_bas = p.basis + dm.basis_offset;
    const bool grouped = N >= 32 || !shape_pow2(N);
    const uint32_t pairs = shape_any_pairs(N);
    for (uint32_t i = threadIdx.x; i < dm.E * brow; i += THREADS) {
      const uint32_t k = i / brow, r = i - k * brow;
      const uint32_t n = grouped ? 16 * (r / 20) + r % 20 : r;
      const bool in = grouped ? r % 20 < 16 && n < pairs : r < half;
      bas[i] = in ? __ldg(g_bas + (size_t)k * N + n) : 0.0f;
    }
  }
  return off;
}

// Where the transform of a tile writes: the warp's staging tile and its row
// of it, the output tensor map, and whether a TMA store is still reading it.
struct ShapeOut {
  unsigned char *otile;
  unsigned char *row;
  uint32_t sx;
  uint32_t lane;
  const CUtensorMap *map;
  bool tma_ok;  // the segment's output starts on a 128-byte boundary and the map is valid
  bool vec32, vec16;
};

// Dequantization + inverse transform + reassembly of one decoded tile of nwin
// windows (levels at stage[0..nwin E)), 1024 samples per step.
template <int N>
__device__ __forceinline__ void shape_transform(const DecodeParams &p, const SegDev &sg, const DomS &dd,
                                                const unsigned char *smem, const uint8_t *stage, uint64_t win0,
                                                uint32_t nwin, const ShapeOut &o, bool &tma_pending) {
  using K = ShapeK<N>;
  const uint32_t lane = o.lane;
  const float *deq0 = reinterpret_cast<const float *>(smem + dd.deq_off);
  const float *bas = reinterpret_cast<const float *>(smem + dd.basis_off);
  const uint64_t S = sg.n_samples;
#pragma unroll 1
  for (uint32_t w0 = 0; w0 < nwin; w0 += K::R) {
    const bool tma_step = o.tma_ok && w0 + K::R <= nwin && (win0 + w0 + K::R) * N <= S;
    if (tma_pending) {
      if (lane == 0) tma_wait_read();  // the previous step has left the staging tile
      __syncwarp();
      tma_pending = false;
    }
    float ev[16], od[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) ev[i] = od[i] = 0.0f;
    if (N >= 32) {
      const uint32_t wl = w0 + lane / K::L, q = lane % K::L;
      if (wl < nwin) {
        const uint8_t *lv = stage + wl * dd.E;
        const float *bq = bas + q * 20;
        uint32_t k = 0;
#pragma unroll 1
        for (; k + 2 <= dd.kz; k += 2) {
          const float c0 = deq0[(k < dd.B1 ? 0 : kZStride) + lv[k]];
          const float c1 = deq0[(k + 1 < dd.B1 ? 0 : kZStride) + lv[k + 1]];
          const float4 *b0 = reinterpret_cast<const float4 *>(bq + k * K::BROW);
          const float4 *b1 = reinterpret_cast<const float4 *>(bq + (k + 1) * K::BROW);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 u = b0[j], v = b1[j];
            ev[4 * j] = fmaf(c0, u.x, ev[4 * j]);
            ev[4 * j + 1] = fmaf(c0, u.y, ev[4 * j + 1]);
            ev[4 * j + 2] = fmaf(c0, u.z, ev[4 * j + 2]);
            ev[4 * j + 3] = fmaf(c0, u.w, ev[4 * j + 3]);
            od[4 * j] = fmaf(c1, v.x, od[4 * j]);
            od[4 * j + 1] = fmaf(c1, v.y, od[4 * j + 1]);
            od[4 * j + 2] = fmaf(c1, v.z, od[4 * j + 2]);
            od[4 * j + 3] = fmaf(c1, v.w, od[4 * j + 3]);
          }
        }
        if (k < dd.kz) {  // a last even bin
          const float c0 = deq0[(k < dd.B1 ? 0 : kZStride) + lv[k]];
          const float4 *b0 = reinterpret_cast<const float4 *>(bq + k * K::BROW);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 u = b0[j];
            ev[4 * j] = fmaf(c0, u.x, ev[4 * j]);
            ev[4 * j + 1] = fmaf(c0, u.y, ev[4 * j + 1]);
            ev[4 * j + 2] = fmaf(c0, u.z, ev[4 * j + 2]);
            ev[4 * j + 3] = fmaf(c0, u.w, ev[4 * j + 3]);
          }
        }
      }
      // samples 16 q .. 16 q + 15 of the window and their mirrors, at step
      // positions (lane / L) N + ...: two half rows of the staging tile
      const uint32_t base = (lane / K::L) * N;
      const uint32_t f0 = base + 16 * q, m0 = base + N - 16 * (q + 1);
      float xf[16], xm[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        xf[i] = ev[i] + od[i];
        xm[15 - i] = ev[i] - od[i];
      }
      unsigned char *const rf = o.otile + (f0 >> 5) * 128;
      unsigned char *const rm = o.otile + (m0 >> 5) * 128;
      const uint32_t cf = (f0 & 31u) >> 2, cm = (m0 & 31u) >> 2;
      const uint32_t sf = (f0 >> 5) & 7u, sm = (m0 >> 5) & 7u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        *reinterpret_cast<float4 *>(rf + (((cf + j) ^ sf) << 4)) =
            make_float4(xf[4 * j], xf[4 * j + 1], xf[4 * j + 2], xf[4 * j + 3]);
        *reinterpret_cast<float4 *>(rm + (((cm + j) ^ sm) << 4)) =
            make_float4(xm[4 * j], xm[4 * j + 1], xm[4 * j + 2], xm[4 * j + 3]);
      }
    } else {
      // windows w0 + M lane + j, j < M: their pairs n < P
      const uint32_t wl = w0 + K::M * lane;
#pragma unroll 1
      for (uint32_t k = 0; k < dd.kz; ++k) {
        const float *dq = deq0 + (k < dd.B1 ? 0 : kZStride);
        float b[K::P];
#pragma unroll
        for (int i = 0; i < K::P; i += 4) {
          const float4 u = *reinterpret_cast<const float4 *>(bas + k * K::BROW + i);
          b[i] = u.x;
          if (i + 1 < K::P) b[i + 1] = u.y;
          if (i + 2 < K::P) b[i + 2] = u.z;
          if (i + 3 < K::P) b[i + 3] = u.w;
        }
#pragma unroll
        for (int j = 0; j < K::M; ++j) {
          const float c = wl + j < nwin ? dq[stage[(wl + j) * dd.E + k]] : 0.0f;
#pragma unroll
          for (int i = 0; i < K::P; ++i) {
            if (k & 1u)
              od[j * K::P + i] = fmaf(c, b[i], od[j * K::P + i]);
            else
              ev[j * K::P + i] = fmaf(c, b[i], ev[j * K::P + i]);
          }
        }
      }
      // the lane's row: windows j at positions j N .. j N + N - 1
      float x[32];
#pragma unroll
      for (int j = 0; j < K::M; ++j)
#pragma unroll
        for (int i = 0; i < K::P; ++i) {
          x[j * N + i] = ev[j * K::P + i] + od[j * K::P + i];
          x[j * N + N - 1 - i] = ev[j * K::P + i] - od[j * K::P + i];
        }
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4 *>(o.row + ((c ^ o.sx) << 4)) =
            make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
    }
    const uint64_t s0 = (win0 + w0) * N;  // first sample of the step in the segment
    if (tma_step) {
      fence_async_shared();
      __syncwarp();
      if (lane == 0) tma_store_rows(o.map, o.otile, (int32_t)((sg.out_offset + s0) >> 5));
      tma_pending = true;
    } else {
      __syncwarp();  // rows are written by other lanes
      const uint64_t lim = (uint64_t)(nwin - w0) * N < S - s0 ? (uint64_t)(nwin - w0) * N : S - s0;
      const uint64_t r0 = (uint64_t)lane * 32;
      if (r0 < lim) {
        const uint32_t m = lim - r0 < 32 ? (uint32_t)(lim - r0) : 32u;
        store_row(o.row, o.sx, p.out + sg.out_offset + s0 + r0, m, o.vec32, o.vec16);
      }
      __syncwarp();  // before the next step rewrites the tile
    }
  }
}

// The same for a window size N that is not a power of two (run-time N): a
// window's ceil(N / 2) sample pairs (n, N - 1 - n) in groups of 16, one lane per
// group; a step holds R = min(32 / groups, 1024 / N) windows, R N samples of the
// tile from the staging tile's start, which the lanes store row by row (vector
// stores where a row's address allows).
__device__ __forceinline__ void shape_transform_any(const DecodeParams &p, const SegDev &sg, const DomS &dd,
                                                    const unsigned char *smem, const uint8_t *stage, uint64_t win0,
                                                    uint32_t nwin, const ShapeOut &o, bool &tma_pending) {
  const uint32_t N = dd.N, P = shape_any_pairs(N), L = shape_any_lanes(N), R = shape_any_step(N);
  const uint32_t brow = L * 20u;
  const uint32_t lane = o.lane;
  const float *deq0 = reinterpret_cast<const float *>(smem + dd.deq_off);
  const float *bas = reinterpret_cast<const float *>(smem + dd.basis_off);
  const uint64_t S = sg.n_samples;
  if (tma_pending) {  // a previous tile's TMA store may still read the staging tile
    if (lane == 0) tma_wait_read();
    __syncwarp();
    tma_pending = false;
  }
  const uint32_t wr = lane / L, q = lane % L;  // window of the step, pair group
#pragma unroll 1
  for (uint32_t w0 = 0; w0 < nwin; w0 += R) {
    const uint32_t wl = w0 + wr;
    const bool mine = wr < R && wl < nwin;
    float ev[16], od[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) ev[i] = od[i] = 0.0f;
    if (mine) {
      const uint8_t *lv = stage + wl * dd.E;
      const float *bq = bas + q * 20;
      uint32_t k = 0;
#pragma unroll 1
      for (; k + 2 <= dd.kz; k += 2) {
        const float c0 = deq0[(k < dd.B1 ? 0 : kZStride) + lv[k]];
        const float c1 = deq0[(k + 1 < dd.B1 ? 0 : kZStride) + lv[k + 1]];
        const float4 *b0 = reinterpret_cast<const float4 *>(bq + k * brow);
        const float4 *b1 = reinterpret_cast<const float4 *>(bq + (k + 1) * brow);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 u = b0[j], v = b1[j];
          ev[4 * j] = fmaf(c0, u.x, ev[4 * j]);
          ev[4 * j + 1] = fmaf(c0, u.y, ev[4 * j + 1]);
          ev[4 * j + 2] = fmaf(c0, u.z, ev[4 * j + 2]);
          ev[4 * j + 3] = fmaf(c0, u.w, ev[4 * j + 3]);
          od[4 * j] = fmaf(c1, v.x, od[4 * j]);
          od[4 * j + 1] = fmaf(c1, v.y, od[4 * j + 1]);
          od[4 * j + 2] = fmaf(c1, v.z, od[4 * j + 2]);
          od[4 * j + 3] = fmaf(c1, v.w, od[4 * j + 3]);
        }
      }
      if (k < dd.kz) {  // a last even bin
        const float c0 = deq0[(k < dd.B1 ? 0 : kZStride) + lv[k]];
        const float4 *b0 = reinterpret_cast<const float4 *>(bq + k * brow);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 u = b0[j];
          ev[4 * j] = fmaf(c0, u.x, ev[4 * j]);
          ev[4 * j + 1] = fmaf(c0, u.y, ev[4 * j + 1]);
          ev[4 * j + 2] = fmaf(c0, u.z, ev[4 * j + 2]);
          ev[4 * j + 3] = fmaf(c0, u.w, ev[4 * j + 3]);
        }
      }
      // samples n = 16 q + i and N - 1 - n of window wr at step positions wr N + ...
      // (the middle sample of an odd N once: its odd-bin basis values are zero)
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const uint32_t n = 16 * q + i;
        if (n < P) {
          const uint32_t tf = wr * N + n, tm = wr * N + (N - 1 - n);
          *reinterpret_cast<float *>(o.otile + (tf >> 5) * 128 + ((((tf & 31u) >> 2) ^ ((tf >> 5) & 7u)) << 4) +
                                     ((tf & 3u) << 2)) = ev[i] + od[i];
          if (tm != tf)
            *reinterpret_cast<float *>(o.otile + (tm >> 5) * 128 + ((((tm & 31u) >> 2) ^ ((tm >> 5) & 7u)) << 4) +
                                       ((tm & 3u) << 2)) = ev[i] - od[i];
        }
      }
    }
    __syncwarp();  // rows are written by other lanes
    const uint64_t s0 = (win0 + w0) * N;  // first sample of the step in the segment
    const uint32_t nw = nwin - w0 < R ? nwin - w0 : R;
    const uint64_t lim = (uint64_t)nw * N < S - s0 ? (uint64_t)nw * N : S - s0;
    const uint64_t r0 = (uint64_t)lane * 32;
    if (r0 < lim) {
      const uint32_t m = lim - r0 < 32 ? (uint32_t)(lim - r0) : 32u;
      float *const dst = p.out + sg.out_offset + s0 + r0;
      const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
      store_row(o.row, o.sx, dst, m, (a & 31u) == 0, (a & 15u) == 0);
    }
    __syncwarp();  // before the next step rewrites the tile
  }
}

// ANY: a domain of the plan has a window size that is not a power of two (its
// transform is compiled only into this instance, whose registers it costs).
template <int WARPS, bool ANY>
__global__ void __launch_bounds__(WARPS * 32, 1) k_decode_shape(const DecodeParams p, const WarpParams wp,
                                                                const __grid_constant__ CUtensorMap out_map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DomS *const ds = reinterpret_cast<const DomS *>(smem_raw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  load_shape_tables<WARPS * 32>(p, wp.n_domains, smem_raw);
  __syncthreads();

  unsigned char *const wbase = smem_raw + wp.warp_off + warp * kMiscBytes;
  uint64_t *const wbuf = reinterpret_cast<uint64_t *>(wbase);  // first-pass words
  uint8_t *const stage = wbase + kStageOff;      // tile position 0
  const uintptr_t tiles0 = (reinterpret_cast<uintptr_t>(smem_raw + wp.warp_off + WARPS * kMiscBytes) + 1023) &
                           ~uintptr_t(1023);
  unsigned char *const otile = reinterpret_cast<unsigned char *>(tiles0) + warp * kOutTile;
  unsigned char *const row = otile + lane * 128;  // this lane's row of the staging tile
  const uint32_t sx = lane & 7u;
  const bool want_lev = p.levels != nullptr;
  bool tma_pending = false;

  uint64_t tw0, tw1;
  unit_tiles(p, (uint64_t)blockIdx.x * WARPS + warp, (uint64_t)gridDim.x * WARPS, tw0, tw1);
  if (tw0 >= tw1) return;

  Ctx nxt;
  {
    const uint32_t s = find_segment(p.segs, p.seg_begin, p.seg_end, tw0);
    const DomS &d0 = ds[p.segs[s].domain];
    nxt = first_ctx(p, s, tw0, lane, (uint64_t)d0.T * d0.E);
  }
  uint32_t pn = fetch_pass0(p, nxt, lane, wbuf);

  for (uint64_t g = tw0; g < tw1; ++g) {
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
    const DomS dd = ds[sg.domain];
    const uint64_t win0 = (g - sg.tile_base) * dd.T;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = left < (uint64_t)dd.T ? (uint32_t)left : dd.T;

    // ---- 1. SymLen decode into the level bytes
    TileEnd te{0u, 0u, 0u};
    if (cur.ok) {
      te = decode_tile(p, cur, nwin * dd.E, dd, smem_raw, stage, lane, w, n);
      if (te.bad && lane == 0) flag_bad(p.status, te.bad, sg.caller_index);
    }
    // ---- first words of tile g + 1 (in flight during the transform)
    if (g1 < tw1) {
      nxt = next_ctx(p, g, cur.seg, cur, te);
      pn = fetch_pass0(p, nxt, lane, wbuf);
    }
    __syncwarp();
    if (!cur.ok) continue;

    if (want_lev) {  // the tile's levels are contiguous in the caller's buffer
      uint8_t *const lev = p.levels + sg.level_offset + win0 * dd.E;
      for (uint32_t j = lane; j < nwin * dd.E; j += 32) lev[j] = stage[j];
    }

    // ---- 2./3. dequantization + inverse transform + reassembly, 1024 samples per step
    const uint32_t aligned = sg.out_aligned;
    ShapeOut o{otile, row, sx, lane, &out_map, wp.out_tma && (aligned & 4u),
               (aligned & 2u) && (reinterpret_cast<uintptr_t>(p.out) & 31u) == 0, (aligned & 1u) != 0};
    switch (dd.N) {  // the tile's domain: uniform over the warp
      case 4: shape_transform<4>(p, sg, dd, smem_raw, stage, win0, nwin, o, tma_pending); break;
      case 8: shape_transform<8>(p, sg, dd, smem_raw, stage, win0, nwin, o, tma_pending); break;
      case 16: shape_transform<16>(p, sg, dd, smem_raw, stage, win0, nwin, o, tma_pending); break;
      case 32: shape_transform<32>(p, sg, dd, smem_raw, stage, win0, nwin, o, tma_pending); break;
      case 64: shape_transform<64>(p, sg, dd, smem_raw, stage, win0, nwin, o, tma_pending); break;
      case 128: shape_transform<128>(p, sg, dd, smem_raw, stage, win0, nwin, o, tma_pending); break;
      default:
        if (ANY) shape_transform_any(p, sg, dd, smem_raw, stage, win0, nwin, o, tma_pending);
        break;
    }
    __syncwarp();  // the level bytes are rewritten by the next tile
  }
  if (tma_pending && lane == 0) tma_wait_all();
}

void *spick(uint32_t threads, bool any) {
  switch (threads) {
    case 256: return any ? reinterpret_cast<void *>(&k_decode_shape<8, true>) : reinterpret_cast<void *>(&k_decode_shape<8, false>);
    case 512: return any ? reinterpret_cast<void *>(&k_decode_shape<16, true>) : reinterpret_cast<void *>(&k_decode_shape<16, false>);
    case 768: return any ? reinterpret_cast<void *>(&k_decode_shape<24, true>) : reinterpret_cast<void *>(&k_decode_shape<24, false>);
    default: return nullptr;
  }
}

}  // namespace

bool shape_supported(uint32_t N) { return N >= 4 && N <= 128; }

bool shape_pow2_only(uint32_t N) { return shape_pow2(N); }

uint32_t shape_windows_per_tile(uint32_t N, uint32_t E) { return shape_tile_windows(N, E); }

size_t shape_smem_layout(uint32_t threads, const uint32_t *lmax, const uint32_t *N, const uint32_t *E,
                         uint32_t n_domains, WarpParams *wp) {
  size_t o = align16(sizeof(DomS) * (n_domains ? n_domains : 1));
  for (uint32_t d = 0; d < n_domains; ++d) {
    o += align16((size_t)2 << lmax[d]);
    o += align16(3u * kZStride * 4);
    o += align16((size_t)E[d] * shape_brow(N[d]) * 4);
  }
  o = align16(o);
  *wp = WarpParams{};
  wp->n_domains = n_domains;
  wp->warp_off = (uint32_t)o;
  wp->warp_bytes = (uint32_t)kMiscBytes;
  const size_t warps = threads / 32;
  return o + warps * kMiscBytes + 1023 + warps * kOutTile;  // + alignment of the staging tiles
}

cudaError_t shape_smem_config(uint32_t threads, bool any, size_t smem) {
  void *k = spick(threads, any);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return set_dynamic_smem_limit(k, smem);
}

cudaError_t shape_occupancy(uint32_t threads, bool any, size_t smem, int *ctas_per_sm) {
  void *k = spick(threads, any);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, (int)threads, smem);
}

cudaError_t launch_shape(const DecodeParams &p, const WarpParams &wp, const CUtensorMap &out_map, uint32_t threads,
                         bool any, uint32_t grid, size_t smem, cudaStream_t stream) {
  if (p.tile_end <= p.tile_begin || grid == 0) return cudaSuccess;
  void *k = spick(threads, any);
  if (!k) return cudaErrorInvalidValue;
  DecodeParams pp = p;
  WarpParams ww = wp;
  CUtensorMap mm = out_map;
  void *args[] = {&pp, &ww, &mm};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
