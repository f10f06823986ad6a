// Fused FPTC decode (Sec. 4.2): one persistent kernel does, per tile of
// tile_windows windows, what the paper splits into a lossless kernel
// (per-word Huffman decode + compaction, Sec. 4.2.1) and a lossy kernel
// (dequantization + inverse DCT, Sec. 4.2.2):
//   1. the tile's SymLen words are decoded one word per thread with the
//      decode table in shared memory; a block scan of symlen places every
//      word's run in the tile, so compaction happens in shared memory
//      (no global uint8 round trip);
//   2. each symbol is dequantized as it is decoded (table A_z * unit_z(level));
//   3. the inverse transform x[n] = sum_k C[k] B[k][n] (B[0][n] = 1/2) runs
//      per window and the samples go to the segment's output range.
// CTAs take contiguous ranges of the tile queue; a tile's start comes from the
// index kernels, so no CTA waits on another.
//
// Two instantiations: a generic one for any N, E (basis read through L1), and
// a fixed N = 32, E = 16 one that keeps its basis columns in registers, uses the
// mirror symmetry B[k][N-1-n] = (-1)^k B[k][n] to halve the multiply-adds, packs
// them in FFMA2 (two FP32 FMAs per instruction) and stores 16-byte vectors.
#include "device_util.cuh"

namespace fptc {
namespace {

constexpr int kFixedN = 32;
constexpr int kFixedE = 16;

struct Smem {
  uint16_t *lut;
  float *deq;
  float *coef;
  uint8_t *lev;
  uint32_t *scan;
};

__device__ __forceinline__ Smem carve(unsigned char *base, uint32_t lut_cap, uint32_t coef_cap) {
  Smem s;
  size_t o = 0;
  s.lut = reinterpret_cast<uint16_t *>(base + o);
  o += align16((size_t)lut_cap * 2);
  s.deq = reinterpret_cast<float *>(base + o);
  o += 512 * 4;
  s.coef = reinterpret_cast<float *>(base + o);
  o += align16((size_t)coef_cap * 4);
  s.lev = base + o;
  o += align16(coef_cap);
  s.scan = reinterpret_cast<uint32_t *>(base + o);
  return s;
}

template <int THREADS, bool FIXED>
__global__ void __launch_bounds__(THREADS) k_decode(const DecodeParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = carve(smem_raw, p.lut_cap, p.coef_cap);

  const uint64_t n_all = p.tile_end - p.tile_begin;
  const uint64_t t0 = p.tile_begin + n_all * blockIdx.x / gridDim.x;
  const uint64_t t1 = p.tile_begin + n_all * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;

  uint32_t s = find_segment(p.segs, p.seg_begin, p.seg_end, t0);
  uint32_t cur_dom = 0xFFFFFFFFu;
  unsigned int err = 0;

  // FIXED: basis columns n = 4q .. 4q+3 of every bin, as FFMA2 pairs
  constexpr int Q = kFixedN / 8;
  const uint32_t q = threadIdx.x % Q;
  float2 bp[FIXED ? kFixedE : 1][2];

  for (uint64_t g = t0; g < t1; ++g) {
    while (g >= p.segs[s].tile_base + p.segs[s].n_tiles) ++s;
    if (p.seg_bad[s]) continue;  // same value for every thread of the block
    const SegDev sg = p.segs[s];
    const DomainDev &dm = p.domains[sg.domain];
    const uint32_t N = FIXED ? kFixedN : dm.N;
    const uint32_t E = FIXED ? kFixedE : dm.E;
    const uint32_t B1 = dm.B1, B2 = dm.B2, lmax = dm.lmax;
    if (sg.domain != cur_dom) {
      __syncthreads();
      load_lut<THREADS>(sm.lut, p.luts + dm.lut_offset, 1u << lmax);
      load_deq<THREADS>(sm.deq, dm, p.scale, sg.domain);
      if (FIXED) {
        const float *b = p.basis + dm.basis_offset;
#pragma unroll
        for (int k = 0; k < (FIXED ? kFixedE : 1); ++k) {
          bp[k][0] = make_float2(__ldg(b + k * kFixedN + 4 * q), __ldg(b + k * kFixedN + 4 * q + 1));
          bp[k][1] = make_float2(__ldg(b + k * kFixedN + 4 * q + 2), __ldg(b + k * kFixedN + 4 * q + 3));
        }
      }
      cur_dom = sg.domain;
      __syncthreads();
    }

    // ---- 1+2: Huffman decode + compaction + dequantization into shared memory
    const uint64_t tin = g - sg.tile_base;
    const uint64_t win0 = tin * dm.tile_windows;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = left < dm.tile_windows ? (uint32_t)left : dm.tile_windows;
    const uint32_t tsyms = nwin * E;
    const TileRec tr = p.tiles[g];
    uint64_t lw;
    if (tin + 1 < sg.n_tiles) {
      const TileRec nx = p.tiles[g + 1];
      lw = nx.first_word - (nx.skip == 0 ? 1u : 0u);
    } else {
      lw = sg.word_offset + sg.n_words - 1;
    }
    const uint64_t fw = tr.first_word;
    const uint64_t nw = lw >= fw ? lw - fw + 1 : 0;
    int64_t base = -(int64_t)tr.skip;
    const bool want_lev = p.levels != nullptr;
    for (uint64_t c0 = 0; c0 < nw; c0 += THREADS) {
      const uint64_t i = c0 + threadIdx.x;
      uint32_t sl = 0;
      uint64_t wd = 0;
      if (i < nw) {
        sl = __ldg(p.symlen + fw + i);
        wd = __ldg(p.words + fw + i);
      }
      uint32_t total;
      const uint32_t ex = block_exclusive_scan<THREADS>(sl, sm.scan, &total);
      if (sl) {
        const int64_t pos = base + ex;
        if (want_lev)
          err |= decode_word<true, true>(wd, sl, pos, tsyms, sm.lut, lmax, E, B1, B2, sm.deq, sm.coef, sm.lev);
        else
          err |= decode_word<true, false>(wd, sl, pos, tsyms, sm.lut, lmax, E, B1, B2, sm.deq, sm.coef, sm.lev);
      }
      base += total;
      if (base >= (int64_t)tsyms) break;  // uniform
    }
    if (err) {
      flag_bad(p.status, err, sg.caller_index);
      err = 0;
    }
    __syncthreads();

    if (want_lev) {
      uint8_t *dst = p.levels + sg.level_offset + win0 * E;
      for (uint32_t i = threadIdx.x; i < tsyms; i += THREADS) dst[i] = sm.lev[i];
    }

    // ---- 3: inverse transform + window reassembly
    float *out = p.out + sg.out_offset;
    const uint64_t S = sg.n_samples;
    if (FIXED) {
      for (uint32_t wl = threadIdx.x / Q; wl < nwin; wl += THREADS / Q) {
        const float4 *c4 = reinterpret_cast<const float4 *>(sm.coef + wl * kFixedE);
        float2 e0 = make_float2(0.f, 0.f), e1 = e0, o0 = e0, o1 = e0;
#pragma unroll
        for (int kk = 0; kk < kFixedE / 4; ++kk) {
          const float4 c = c4[kk];
          const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y);
          const float2 cz = make_float2(c.z, c.z), cw = make_float2(c.w, c.w);
          e0 = __ffma2_rn(cx, bp[4 * kk][0], e0);
          e1 = __ffma2_rn(cx, bp[4 * kk][1], e1);
          o0 = __ffma2_rn(cy, bp[4 * kk + 1][0], o0);
          o1 = __ffma2_rn(cy, bp[4 * kk + 1][1], o1);
          e0 = __ffma2_rn(cz, bp[4 * kk + 2][0], e0);
          e1 = __ffma2_rn(cz, bp[4 * kk + 2][1], e1);
          o0 = __ffma2_rn(cw, bp[4 * kk + 3][0], o0);
          o1 = __ffma2_rn(cw, bp[4 * kk + 3][1], o1);
        }
        // x[n] = even + odd for n = 4q..4q+3; x[N-1-n] = even - odd
        const float4 lo = make_float4(e0.x + o0.x, e0.y + o0.y, e1.x + o1.x, e1.y + o1.y);
        const float4 hi = make_float4(e1.y - o1.y, e1.x - o1.x, e0.y - o0.y, e0.x - o0.x);
        const uint64_t s0 = (win0 + wl) * kFixedN;
        float *dst = out + s0;
        if (s0 + kFixedN <= S && sg.out_aligned) {
          __stcs(reinterpret_cast<float4 *>(dst + 4 * q), lo);
          __stcs(reinterpret_cast<float4 *>(dst + kFixedN - 4 - 4 * q), hi);
        } else {
          const float lv[4] = {lo.x, lo.y, lo.z, lo.w};
          const float hv[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t n1 = 4 * q + j, n2 = kFixedN - 4 - 4 * q + j;
            if (s0 + n1 < S) dst[n1] = lv[j];
            if (s0 + n2 < S) dst[n2] = hv[j];
          }
        }
      }
    } else {
      const float *bas = p.basis + dm.basis_offset;
      const uint32_t nout = nwin * N;
      for (uint32_t i = threadIdx.x; i < nout; i += THREADS) {
        const uint32_t wl = i / N, n = i - wl * N;
        const float *cw = sm.coef + wl * E;
        float acc = 0.f;
        for (uint32_t k = 0; k < E; ++k) acc = fmaf(cw[k], __ldg(bas + k * N + n), acc);
        const uint64_t si = (win0 + wl) * N + n;
        if (si < S) out[si] = acc;
      }
    }
    __syncthreads();
  }
}

template <int THREADS, bool FIXED>
void *kernel_ptr() {
  return reinterpret_cast<void *>(&k_decode<THREADS, FIXED>);
}

void *pick(int, uint32_t threads) {
  switch (threads) {
    case 128: return kernel_ptr<128, false>();
    case 256: return kernel_ptr<256, false>();
    case 512: return kernel_ptr<512, false>();
    default: return nullptr;
  }
}

}  // namespace

size_t decode_smem_bytes(int, uint32_t threads, uint32_t lut_cap, uint32_t coef_cap) {
  return align16((size_t)lut_cap * 2) + 512 * 4 + align16((size_t)coef_cap * 4) + align16(coef_cap) +
         (size_t)(threads / 32) * 4;
}

cudaError_t decode_smem_config(int kind, uint32_t threads, size_t smem) {
  void *k = pick(kind, threads);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return set_dynamic_smem_limit(k, smem);
}

cudaError_t decode_occupancy(int kind, uint32_t threads, size_t smem, int *ctas_per_sm) {
  void *k = pick(kind, threads);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, (int)threads, smem);
}

cudaError_t launch_decode(const DecodeParams &p, int kind, uint32_t threads, uint32_t grid, size_t smem,
                          cudaStream_t stream) {
  if (p.tile_end <= p.tile_begin || grid == 0) return cudaSuccess;
  void *k = pick(kind, threads);
  if (!k) return cudaErrorInvalidValue;
  DecodeParams pp = p;
  void *args[] = {&pp};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
