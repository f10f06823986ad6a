// Adjoint of the lossy decode stage (dequantize + inverse DCT + window
// reassembly, Sec. 4.2.2) for a loss L with dL/dx = g_x:
//   g_C[w][k] = sum_n g_x[wN + n] B[k][n]      (B[0][n] = 1/2; samples past S are 0)
//   dL/dA_z  = sum over bins k of zone z of g_C[w][k] * unit_z(level[w][k])
// because the reconstruction of zone z is A_z * unit_z(level) (both the mu-law
// expander and the deadzone lattice scale linearly with A_z).
// Per tile: levels come from the saved level buffer or are decoded again
// (same SymLen decode as the forward kernel), g_x is staged in shared memory,
// one thread per (window, bin) does the N-term FP32 dot product against the
// transposed basis, products g_C * unit go to an FP32 partial per thread and
// tile, and partials are accumulated in FP64 (per thread, then per block, then
// one FP64 atomic per block and domain/zone).
#include "device_util.cuh"

namespace fptc {
namespace {

struct BSmem {
  uint16_t *lut;
  float *unit;     // [2][256], zeroed for a switched-off zone
  float *basisT;   // [N][E]
  float *gx;       // tile samples
  uint8_t *lev;
  uint32_t *scan;
  double *red;     // [THREADS/32][2]
};

template <int THREADS>
__device__ __forceinline__ void flush_grad(double acc0, double acc1, double *red, double *grad, uint32_t d) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
    acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
  }
  if (lane == 0) {
    red[2 * warp] = acc0;
    red[2 * warp + 1] = acc1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) {
      a += red[2 * w];
      b += red[2 * w + 1];
    }
    if (a != 0.0) atomicAdd(grad + d * 3 + 0, a);
    if (b != 0.0) atomicAdd(grad + d * 3 + 1, b);
  }
  __syncthreads();
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_backward(const BackwardParams bp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DecodeParams &p = bp.d;
  BSmem sm;
  {
    size_t o = 0;
    sm.lut = reinterpret_cast<uint16_t *>(smem_raw + o);
    o += align16((size_t)p.lut_cap * 2);
    sm.unit = reinterpret_cast<float *>(smem_raw + o);
    o += 512 * 4;
    sm.basisT = reinterpret_cast<float *>(smem_raw + o);
    o += align16((size_t)bp.basis_cap * 4);
    sm.gx = reinterpret_cast<float *>(smem_raw + o);
    o += align16((size_t)bp.gx_cap * 4);
    sm.lev = smem_raw + o;
    o += align16(p.coef_cap);
    sm.scan = reinterpret_cast<uint32_t *>(smem_raw + o);
    o += align16((size_t)(THREADS / 32) * 4);
    sm.red = reinterpret_cast<double *>(smem_raw + o);
  }

  const uint64_t n_all = p.tile_end - p.tile_begin;
  const uint64_t t0 = p.tile_begin + n_all * blockIdx.x / gridDim.x;
  const uint64_t t1 = p.tile_begin + n_all * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;

  uint32_t s = find_segment(p.segs, p.seg_begin, p.seg_end, t0);
  uint32_t cur_dom = 0xFFFFFFFFu;
  double acc0 = 0.0, acc1 = 0.0;
  unsigned int err = 0;

  for (uint64_t g = t0; g < t1; ++g) {
    while (g >= p.segs[s].tile_base + p.segs[s].n_tiles) ++s;
    if (p.seg_bad[s] && bp.levels_in == nullptr) continue;
    const SegDev sg = p.segs[s];
    const DomainDev &dm = p.domains[sg.domain];
    const uint32_t N = dm.N, E = dm.E, B1 = dm.B1, B2 = dm.B2, lmax = dm.lmax;
    if (sg.domain != cur_dom) {
      if (cur_dom != 0xFFFFFFFFu) {
        flush_grad<THREADS>(acc0, acc1, sm.red, bp.grad_scale, cur_dom);
        acc0 = acc1 = 0.0;
      }
      __syncthreads();
      if (bp.levels_in == nullptr) load_lut<THREADS>(sm.lut, p.luts + dm.lut_offset, 1u << lmax);
      {
        float a0 = p.scale ? p.scale[sg.domain * 3 + 0] : dm.scale[0];
        float a1 = p.scale ? p.scale[sg.domain * 3 + 1] : dm.scale[1];
        for (uint32_t i = threadIdx.x; i < 512u; i += THREADS) {
          const uint32_t z = i >> 8;
          const bool on = (z == 0 ? a0 : a1) > 1e-30f;
          sm.unit[i] = on ? dm.unit[z][i & 255u] : 0.0f;
        }
      }
      const float *b = p.basis + dm.basis_offset;
      for (uint32_t i = threadIdx.x; i < N * E; i += THREADS) {
        const uint32_t n = i / E, k = i - n * E;
        sm.basisT[i] = __ldg(b + k * N + n);
      }
      cur_dom = sg.domain;
      __syncthreads();
    }

    const uint64_t tin = g - sg.tile_base;
    const uint64_t win0 = tin * dm.tile_windows;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = left < dm.tile_windows ? (uint32_t)left : dm.tile_windows;
    const uint32_t tsyms = nwin * E;

    // levels of the tile
    if (bp.levels_in) {
      const uint8_t *src = bp.levels_in + sg.level_offset + win0 * E;
      for (uint32_t i = threadIdx.x; i < tsyms; i += THREADS) sm.lev[i] = src[i];
    } else {
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
        if (sl)
          err |= decode_word<false, true>(wd, sl, base + ex, tsyms, sm.lut, lmax, E, B1, B2, nullptr, nullptr,
                                          sm.lev);
        base += total;
        if (base >= (int64_t)tsyms) break;
      }
      if (err) {
        flag_bad(p.status, err, sg.caller_index);
        err = 0;
      }
    }
    // g_x of the tile (0 past S)
    const uint64_t s_begin = win0 * N;
    const uint32_t nsmp = nwin * N;
    const float *gsrc = bp.grad_out + sg.out_offset + s_begin;
    for (uint32_t i = threadIdx.x; i < nsmp; i += THREADS) sm.gx[i] = (s_begin + i < sg.n_samples) ? gsrc[i] : 0.0f;
    __syncthreads();

    float part0 = 0.0f, part1 = 0.0f;
    float *gco = bp.grad_coeffs ? bp.grad_coeffs + sg.level_offset + win0 * E : nullptr;
    for (uint32_t i = threadIdx.x; i < tsyms; i += THREADS) {
      const uint32_t wl = i / E, k = i - wl * E;
      const float *gw = sm.gx + wl * N;
      float acc = 0.0f;
      for (uint32_t n = 0; n < N; ++n) acc = fmaf(gw[n], sm.basisT[n * E + k], acc);
      if (gco) gco[i] = acc;
      const uint32_t z = k < B1 ? 0u : (k < B2 ? 1u : 2u);
      if (z == 0)
        part0 = fmaf(acc, sm.unit[sm.lev[i]], part0);
      else if (z == 1)
        part1 = fmaf(acc, sm.unit[256 + sm.lev[i]], part1);
    }
    acc0 += (double)part0;
    acc1 += (double)part1;
    __syncthreads();
  }
  if (cur_dom != 0xFFFFFFFFu) flush_grad<THREADS>(acc0, acc1, sm.red, bp.grad_scale, cur_dom);
}

void *pick(uint32_t threads) {
  switch (threads) {
    case 128: return reinterpret_cast<void *>(&k_backward<128>);
    case 256: return reinterpret_cast<void *>(&k_backward<256>);
    case 512: return reinterpret_cast<void *>(&k_backward<512>);
    default: return nullptr;
  }
}

}  // namespace

size_t backward_smem_bytes(uint32_t threads, uint32_t lut_cap, uint32_t coef_cap, uint32_t gx_cap,
                           uint32_t basis_cap) {
  return align16((size_t)lut_cap * 2) + 512 * 4 + align16((size_t)basis_cap * 4) + align16((size_t)gx_cap * 4) +
         align16(coef_cap) + align16((size_t)(threads / 32) * 4) + (size_t)(threads / 32) * 2 * 8;
}

cudaError_t backward_smem_config(uint32_t threads, size_t smem) {
  void *k = pick(threads);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return set_dynamic_smem_limit(k, smem);
}

cudaError_t backward_occupancy(uint32_t threads, size_t smem, int *ctas_per_sm) {
  void *k = pick(threads);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, (int)threads, smem);
}

cudaError_t launch_backward(const BackwardParams &p, uint32_t threads, uint32_t grid, size_t smem,
                            cudaStream_t stream) {
  if (p.d.tile_end <= p.d.tile_begin || grid == 0) return cudaSuccess;
  void *k = pick(threads);
  if (!k) return cudaErrorInvalidValue;
  BackwardParams pp = p;
  void *args[] = {&pp};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
