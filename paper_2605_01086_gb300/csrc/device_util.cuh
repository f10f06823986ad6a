// Small device helpers shared by the decode and backward kernels.
#pragma once

#include "fptc_internal.h"

namespace fptc {

__device__ __forceinline__ void flag_bad(DevStatus *st, unsigned int flag, uint32_t caller_index) {
  atomicOr(&st->flags, flag);
  atomicMin(&st->first_bad, (unsigned long long)caller_index);
}

// Exclusive scan over a block of THREADS threads; *total = block sum.
// scratch holds THREADS / 32 words.  Contains __syncthreads (call uniformly).
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *scratch, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < THREADS / 32 ? scratch[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < THREADS / 32) scratch[lane] = s;
  }
  __syncthreads();
  const uint32_t before = warp > 0 ? scratch[warp - 1] : 0u;
  *total = scratch[THREADS / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// Segment (queue index) owning global tile g: the last segment whose tile_base <= g.
__device__ __forceinline__ uint32_t find_segment(const SegDev *segs, uint32_t lo, uint32_t hi, uint64_t g) {
  // invariant: answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (segs[mid].tile_base <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Huffman decode of one SymLen word (Sec. 4.2.1): peek lmax bits MSB first,
// look the prefix up in the decode table (entry = level | length << 8), emit,
// shift the word by the code length; exactly n codewords.  The symbol at tile
// position q (q = pos + j) is written when 0 <= q < tsyms; decoding stops once
// q reaches tsyms (the rest of the word belongs to the next tile).  Symbols
// before the tile (q < 0) are decoded only to advance the bit position.
// WRITE_COEF: store the reconstructed coefficient deq[zone][level];
// WRITE_LEV: store the level.  Returns error flags.
template <bool WRITE_COEF, bool WRITE_LEV>
__device__ __forceinline__ unsigned int decode_word(uint64_t wd, uint32_t n, int64_t pos, uint32_t tsyms,
                                                    const uint16_t *__restrict__ lut, uint32_t lmax, uint32_t E,
                                                    uint32_t B1, uint32_t B2, const float *__restrict__ deq,
                                                    float *__restrict__ coef, uint8_t *__restrict__ lev) {
  const uint32_t shift = 64u - lmax;
  uint32_t used = 0;
  uint32_t k = pos > 0 ? (uint32_t)((uint64_t)pos % E) : 0u;
  int64_t q = pos;
  for (uint32_t j = 0; j < n; ++j, ++q) {
    if (q >= (int64_t)tsyms) break;
    const uint32_t e = lut[(uint32_t)(wd >> shift)];
    const uint32_t len = e >> 8;
    if (len == 0) return kFlagInvalidCode;
    used += len;
    if (used > 64u) return kFlagBitOverrun;
    wd <<= len;
    if (q >= 0) {
      const uint32_t sym = e & 0xffu;
      if (WRITE_COEF) {
        const uint32_t z = k < B1 ? 0u : (k < B2 ? 1u : 2u);
        coef[q] = z < 2u ? deq[z * 256u + sym] : 0.0f;
      }
      if (WRITE_LEV) lev[q] = (uint8_t)sym;
      if (++k == E) k = 0;
    }
  }
  return 0u;
}

// Copies a domain's decode table into shared memory (entries = 1 << lmax).
template <int THREADS>
__device__ __forceinline__ void load_lut(uint16_t *s_lut, const uint16_t *__restrict__ g_lut, uint32_t entries) {
  if ((entries & 7u) == 0 && ((reinterpret_cast<uintptr_t>(g_lut) & 15u) == 0)) {
    const uint4 *src = reinterpret_cast<const uint4 *>(g_lut);
    uint4 *dst = reinterpret_cast<uint4 *>(s_lut);
    for (uint32_t i = threadIdx.x; i < entries / 8; i += THREADS) dst[i] = __ldg(src + i);
  } else {
    for (uint32_t i = threadIdx.x; i < entries; i += THREADS) s_lut[i] = __ldg(g_lut + i);
  }
}

// Reconstruction table of the current domain scaled by A_z: deq[z][L] = A_z * unit_z(L).
template <int THREADS>
__device__ __forceinline__ void load_deq(float *s_deq, const DomainDev &dm, const float *run_scale, uint32_t d) {
  float a0 = run_scale ? run_scale[d * 3 + 0] : dm.scale[0];
  float a1 = run_scale ? run_scale[d * 3 + 1] : dm.scale[1];
  a0 = a0 > 1e-30f ? a0 : 0.0f;
  a1 = a1 > 1e-30f ? a1 : 0.0f;
  for (uint32_t i = threadIdx.x; i < 512u; i += THREADS) {
    const uint32_t z = i >> 8;
    s_deq[i] = (z == 0 ? a0 : a1) * dm.unit[z][i & 255u];
  }
}

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// The dynamic shared-memory limit is a per-kernel attribute shared by every plan
// in the process: raise it to the device's opt-in maximum (never lower it to one
// plan's need, which would break the launches of a plan that needs more).
inline cudaError_t set_dynamic_smem_limit(const void *kernel, size_t need) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (need > (size_t)optin) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

}  // namespace fptc
