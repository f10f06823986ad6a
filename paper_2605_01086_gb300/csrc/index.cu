// SymLen segment indexing (Sec. 4.2.1: "an exclusive prefix sum over the symlen
// array ... producing the output offset for each compressed word").
//
// Three small kernels, none of which waits on another CTA:
//   1. chunk_count: per chunk of 2048 words, the sum of symlen (and a check
//      that no symlen exceeds 64);
//   2. segment_scan: one warp per segment scans its chunk sums into chunk
//      offsets and checks the segment total against W*E;
//   3. tile_index: per chunk, a block scan gives every word's symbol offset;
//      every word that holds the first symbol of a tile (tile = tile_windows
//      windows = tile_windows * E symbols) writes (word, symbols to skip).
// The decode kernel then starts each tile without decoding earlier words.
#include "fptc_internal.h"

namespace fptc {
namespace {

__device__ __forceinline__ void flag_bad(DevStatus *st, unsigned int flag, uint32_t caller_index) {
  atomicOr(&st->flags, flag);
  atomicMin(&st->first_bad, (unsigned long long)caller_index);
}

template <int THREADS>
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) t += scratch[w];
  __syncthreads();
  return t;
}

// exclusive scan over the block; returns the exclusive prefix, *total the sum
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
    if (lane < THREADS / 32) scratch[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  uint32_t before = warp > 0 ? scratch[warp - 1] : 0u;
  *total = scratch[THREADS / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kIndexThreads) k_chunk_count(IndexParams p) {
  __shared__ uint32_t scratch[kIndexThreads / 32];
  const uint64_t c = p.chunk_begin + blockIdx.x;
  if (c >= p.chunk_end) return;
  const ChunkDev ch = p.chunks[c];
  uint32_t sum = 0, bad = 0;
  for (uint32_t i = threadIdx.x; i < ch.n_words; i += kIndexThreads) {
    uint32_t v = p.symlen[ch.word_begin + i];
    bad |= v > 64u;
    sum += v;
  }
  sum = block_sum<kIndexThreads>(sum, scratch);
  bad = block_sum<kIndexThreads>(bad, scratch);
  if (threadIdx.x == 0) p.chunk_sum[c] = bad ? kChunkBad : sum;
}

// one warp per segment
__global__ void __launch_bounds__(256) k_segment_scan(IndexParams p) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t s = (uint64_t)p.seg_begin + (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32;
  if (s >= p.seg_end) return;
  const SegDev sg = p.segs[s];
  uint64_t run = 0;
  bool range_bad = false;
  for (uint32_t j0 = 0; j0 < sg.n_chunks; j0 += 32) {
    const uint32_t j = j0 + lane;
    uint32_t v = j < sg.n_chunks ? p.chunk_sum[sg.chunk_base + j] : 0u;
    if (v == kChunkBad) {
      range_bad = true;
      v = 0;
    }
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (j < sg.n_chunks) p.chunk_off[sg.chunk_base + j] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  range_bad = __any_sync(0xffffffffu, range_bad);
  const uint64_t expect = sg.n_windows * (uint64_t)p.domains[sg.domain].E;
  const bool count_bad = run != expect;
  if (lane == 0) {
    p.seg_bad[s] = (range_bad || count_bad) ? 1u : 0u;
    if (range_bad) flag_bad(p.status, kFlagSymlenRange, sg.caller_index);
    if (count_bad) flag_bad(p.status, kFlagSymbolCount, sg.caller_index);
  }
}

__global__ void __launch_bounds__(kIndexThreads) k_tile_index(IndexParams p) {
  __shared__ uint32_t scratch[kIndexThreads / 32];
  constexpr uint32_t kPer = kChunkWords / kIndexThreads;
  const uint64_t c = p.chunk_begin + blockIdx.x;
  if (c >= p.chunk_end) return;
  const ChunkDev ch = p.chunks[c];
  if (p.seg_bad[ch.seg]) return;  // uniform over the block
  const SegDev sg = p.segs[ch.seg];
  const DomainDev &dm = p.domains[sg.domain];
  const uint64_t te = (uint64_t)dm.tile_windows * dm.E;  // symbols per tile

  const uint32_t i0 = threadIdx.x * kPer;
  uint32_t v[kPer];
  uint32_t tsum = 0;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    v[j] = (i0 + j) < ch.n_words ? (uint32_t)p.symlen[ch.word_begin + i0 + j] : 0u;
    tsum += v[j];
  }
  uint32_t total;
  const uint32_t ex = block_exclusive_scan<kIndexThreads>(tsum, scratch, &total);
  if (tsum == 0) return;
  uint64_t off = p.chunk_off[c] + ex;  // symbol offset (in the segment) of word i0
  // first tile whose start is >= off
  uint64_t tn, ns;
  if (off < 0xFFFFFFFFull && te < 0xFFFFFFFFull) {
    const uint32_t o32 = (uint32_t)off, t32 = (uint32_t)te;
    tn = (o32 + t32 - 1u) / t32;
  } else {
    tn = (off + te - 1) / te;
  }
  ns = tn * te;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    const uint64_t end = off + v[j];
    while (ns < end) {
      if (tn < sg.n_tiles) {
        TileRec r;
        r.first_word = ch.word_begin + i0 + j;
        r.skip = (uint32_t)(ns - off);
        r.pad = 0;
        p.tiles[sg.tile_base + tn] = r;
      }
      ++tn;
      ns += te;
    }
    off = end;
  }
}

}  // namespace

cudaError_t launch_index(const IndexParams &p, cudaStream_t stream) {
  const uint64_t n_chunks = p.chunk_end - p.chunk_begin;
  const uint32_t n_segs = p.seg_end - p.seg_begin;
  if (n_segs == 0) return cudaSuccess;
  if (n_chunks > 0) {
    if (n_chunks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    k_chunk_count<<<(unsigned)n_chunks, kIndexThreads, 0, stream>>>(p);
  }
  const uint64_t warps_threads = (uint64_t)n_segs * 32;
  k_segment_scan<<<(unsigned)((warps_threads + 255) / 256), 256, 0, stream>>>(p);
  if (n_chunks > 0) k_tile_index<<<(unsigned)n_chunks, kIndexThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace fptc
