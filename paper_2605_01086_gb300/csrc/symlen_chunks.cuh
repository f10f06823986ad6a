// Geometry of the index chunks over a segment's symlen bytes (Sec. 4.2.1: the
// symbol offset of a SymLen word is the sum of the symlen of the words before
// it), shared by the index kernels and the decode kernels that locate their
// first tile themselves.
//
// A segment's symlen bytes are cut at 16-byte boundaries of the address space:
// with A the first boundary at or after the segment's first byte, block b
// covers [A + 16 b, A + 16 b + 16), b >= -1, and chunk k is blocks
// 31 k - 1 .. 31 k + 29, one per lane (lane 31 idles).  Every block but the
// segment's first and last lies inside the segment and is read with one
// 16-byte load; those two are read byte by byte, so nothing outside the
// segment is read.
#pragma once

#include "fptc_internal.h"

namespace fptc {

static_assert(kChunkWords == 31 * 16, "a chunk is 31 blocks of 16 bytes");

// A lane's view of one chunk: its 16 symlen bytes (zero outside the segment)
// and the global word index of byte 0 of its block.
struct LaneBlock {
  uint4 v;
  uint64_t word0;
};

// Block 31 k - 1 + lane of segment sg (lane < 31).
__device__ __forceinline__ LaneBlock load_block(const uint8_t *symlen, const SegDev &sg, uint64_t k, uint32_t lane) {
  LaneBlock r;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(symlen + sg.word_offset);
  const uintptr_t a1 = a0 + sg.n_words;
  const uintptr_t blk = ((a0 + 15) & ~uintptr_t(15)) + 16 * (uintptr_t)(31 * k + lane) - 16;
  r.word0 = sg.word_offset + (uint64_t)(blk - a0);  // wraps below word_offset for block -1 (masked bytes)
  if (lane < 31 && blk >= a0 && blk + 16 <= a1) {
    r.v = __ldg(reinterpret_cast<const uint4 *>(blk));
  } else {
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (lane < 31 && blk + 16 > a0 && blk < a1) {  // the segment's first or last block
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uintptr_t a = blk + j;
        if (a >= a0 && a < a1) w[j >> 2] |= (uint32_t)__ldg(reinterpret_cast<const uint8_t *>(a)) << (8 * (j & 3));
      }
    }
    r.v = make_uint4(w[0], w[1], w[2], w[3]);
  }
  return r;
}

__device__ __forceinline__ uint32_t block_sum(const uint4 &v) {
  uint32_t s = __dp4a(v.x, 0x01010101u, 0u);
  s = __dp4a(v.y, 0x01010101u, s);
  s = __dp4a(v.z, 0x01010101u, s);
  return __dp4a(v.w, 0x01010101u, s);
}

__device__ __forceinline__ bool block_over64(const uint4 &v) {
  const uint32_t t = 0x40404040u;
  return (__vcmpgtu4(v.x, t) | __vcmpgtu4(v.y, t) | __vcmpgtu4(v.z, t) | __vcmpgtu4(v.w, t)) != 0u;
}

// The word of segment sg that holds symbol `target` (< the segment's symbol
// count) and how many of its symbols come before it, from the chunk offsets of
// the index (chunk_off[c] = symbol offset in the segment of chunk c's first
// word): the last chunk whose offset is <= target, by binary search, then a
// warp scan over that chunk's blocks.  Warp-collective; every lane gets the
// result.
__device__ __forceinline__ TileRec symbol_word(const uint8_t *symlen, const uint64_t *chunk_off, const SegDev &sg,
                                               uint64_t target, uint32_t lane) {
  uint64_t lo = sg.chunk_base, hi = sg.chunk_base + sg.n_chunks;
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (chunk_off[mid] <= target)
      lo = mid;
    else
      hi = mid;
  }
  const LaneBlock b = load_block(symlen, sg, lo - sg.chunk_base, lane);
  const uint32_t tsum = block_sum(b.v);
  uint32_t x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  uint64_t off = chunk_off[lo] + (x - tsum);  // symbol offset of the block's first word
  uint32_t hit = 0u, j_hit = 0u, skip = 0u;
  if (tsum != 0 && off <= target && target < off + tsum) {
    const uint32_t wv[4] = {b.v.x, b.v.y, b.v.z, b.v.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint64_t end = off + ((wv[j >> 2] >> (8 * (j & 3))) & 0xffu);
      if (!hit && target < end) {
        hit = 1u;
        j_hit = (uint32_t)j;
        skip = (uint32_t)(target - off);
      }
      off = end;
    }
  }
  const uint32_t m = __ballot_sync(0xffffffffu, hit);
  const uint32_t src = m ? (uint32_t)(__ffs(m) - 1) : 0u;
  TileRec r;
  r.first_word = __shfl_sync(0xffffffffu, b.word0 + j_hit, src);
  r.skip = __shfl_sync(0xffffffffu, skip, src);
  r.pad = m ? 0u : 1u;  // 1: not found (inconsistent offsets)
  return r;
}

}  // namespace fptc
