// SymLen segment indexing (Sec. 4.2.1: an exclusive prefix sum over the symlen
// array gives every compressed word the output position of its first symbol).
//
// Three kernels, none of which waits on another CTA:
//   1. chunk_count: per chunk of kChunkWords words, the sum of symlen (and a
//      check that no symlen exceeds 64);
//   2. segment_scan: one warp per segment scans its chunk sums into chunk
//      offsets and checks the segment total against W*E;
//   3. tile_index: per chunk, a warp scan gives every word's symbol offset;
//      every word that holds the first symbol of a tile (tile = tile_windows
//      windows = tile_windows * E symbols) writes (word, symbols to skip).
// The decode kernels then start each tile without decoding earlier words.
//
// Kernels 1 and 3 run one warp per chunk over a contiguous chunk range per
// warp (the segment cursor advances with the chunk index, so no per-chunk
// table is read).  A segment's symlen bytes are cut at 16-byte boundaries of
// the address space: with A the first boundary at or after the segment's
// first byte, block b covers [A + 16 b, A + 16 b + 16), b >= -1, and chunk k
// is blocks 31 k - 1 .. 31 k + 29, one per lane (lane 31 idles).  Every block
// but the segment's first and last lies inside the segment and is read with
// one 16-byte load; those two are read byte by byte, so nothing outside the
// segment is read.  The next chunk's block is loaded while the current one is
// reduced.
#include "fptc_internal.h"

namespace fptc {
namespace {

static_assert(kChunkWords == 31 * 16, "a chunk is 31 blocks of 16 bytes");

__device__ __forceinline__ void flag_bad(DevStatus *st, unsigned int flag, uint32_t caller_index) {
  atomicOr(&st->flags, flag);
  atomicMin(&st->first_bad, (unsigned long long)caller_index);
}

// Segment (queue index) owning chunk c: the last segment whose chunk_base <= c.
__device__ __forceinline__ uint32_t chunk_segment(const SegDev *segs, uint32_t lo, uint32_t hi, uint64_t c) {
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (segs[mid].chunk_base <= c)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

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

// This warp's chunk range [c0, c1) of the launch.
__device__ __forceinline__ void warp_chunks(const IndexParams &p, uint64_t &c0, uint64_t &c1) {
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t n = p.chunk_end - p.chunk_begin;
  c0 = p.chunk_begin + n * gw / nw;
  c1 = p.chunk_begin + n * (gw + 1) / nw;
}

__global__ void __launch_bounds__(256) k_chunk_count(IndexParams p) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t c0, c1;
  warp_chunks(p, c0, c1);
  if (c0 >= c1) return;
  uint32_t s = chunk_segment(p.segs, p.seg_begin, p.seg_end, c0);
  while (c0 >= p.segs[s].chunk_base + p.segs[s].n_chunks) ++s;
  LaneBlock cur = load_block(p.symlen, p.segs[s], c0 - p.segs[s].chunk_base, lane);
  for (uint64_t c = c0; c < c1; ++c) {
    LaneBlock nxt{make_uint4(0u, 0u, 0u, 0u), 0};
    if (c + 1 < c1) {
      while (c + 1 >= p.segs[s].chunk_base + p.segs[s].n_chunks) ++s;
      nxt = load_block(p.symlen, p.segs[s], c + 1 - p.segs[s].chunk_base, lane);
    }
    const uint32_t sum = __reduce_add_sync(0xffffffffu, block_sum(cur.v));
    const uint32_t bad = __reduce_or_sync(0xffffffffu, block_over64(cur.v) ? 1u : 0u);
    if (lane == 0) p.chunk_sum[c] = bad ? kChunkBad : sum;
    cur = nxt;
  }
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

__global__ void __launch_bounds__(256) k_tile_index(IndexParams p) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t c0, c1;
  warp_chunks(p, c0, c1);
  if (c0 >= c1) return;
  uint32_t s = chunk_segment(p.segs, p.seg_begin, p.seg_end, c0);
  while (c0 >= p.segs[s].chunk_base + p.segs[s].n_chunks) ++s;
  LaneBlock cur = load_block(p.symlen, p.segs[s], c0 - p.segs[s].chunk_base, lane);
  uint64_t off_cur = p.chunk_off[c0];
  uint32_t scur = s;
  for (uint64_t c = c0; c < c1; ++c) {
    LaneBlock nxt{make_uint4(0u, 0u, 0u, 0u), 0};
    uint64_t off_nxt = 0;
    uint32_t snxt = s;
    if (c + 1 < c1) {
      while (c + 1 >= p.segs[s].chunk_base + p.segs[s].n_chunks) ++s;
      snxt = s;
      nxt = load_block(p.symlen, p.segs[s], c + 1 - p.segs[s].chunk_base, lane);
      off_nxt = p.chunk_off[c + 1];
    }
    if (p.seg_bad[scur] == 0) {  // uniform over the warp
      const SegDev &sg = p.segs[scur];
      const DomainDev &dm = p.domains[sg.domain];
      const uint64_t te = (uint64_t)dm.tile_windows * dm.E;  // symbols per tile
      const uint32_t tsum = block_sum(cur.v);
      uint32_t x = tsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
      }
      if (tsum) {
        uint64_t off = off_cur + (x - tsum);  // symbol offset (in the segment) of the block's first word
        // first tile whose start is >= off
        uint64_t tn = off < 0xFFFFFFFFull && te < 0xFFFFFFFFull ? ((uint32_t)off + (uint32_t)te - 1u) / (uint32_t)te
                                                                  : (off + te - 1) / te;
        uint64_t ns = tn * te;
        const uint32_t wv[4] = {cur.v.x, cur.v.y, cur.v.z, cur.v.w};
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint64_t end = off + ((wv[j >> 2] >> (8 * (j & 3))) & 0xffu);
          while (ns < end) {
            if (tn < sg.n_tiles) {
              TileRec r;
              r.first_word = cur.word0 + j;
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
    }
    cur = nxt;
    off_cur = off_nxt;
    scur = snxt;
  }
}

// Symbol offset (in the segment) of every word, for the three-kernel schedule
// (Sec. 4.2.1 as the paper runs it: a global array of per-word offsets).
__global__ void __launch_bounds__(256) k_word_offsets(IndexParams p, uint32_t *word_off) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t c0, c1;
  warp_chunks(p, c0, c1);
  if (c0 >= c1) return;
  uint32_t s = chunk_segment(p.segs, p.seg_begin, p.seg_end, c0);
  for (uint64_t c = c0; c < c1; ++c) {
    while (c >= p.segs[s].chunk_base + p.segs[s].n_chunks) ++s;
    const SegDev &sg = p.segs[s];
    const LaneBlock b = load_block(p.symlen, sg, c - sg.chunk_base, lane);
    const uint32_t tsum = block_sum(b.v);
    uint32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (p.seg_bad[s] != 0) continue;  // uniform over the warp
    uint32_t off = (uint32_t)p.chunk_off[c] + (x - tsum);
    const uint32_t wv[4] = {b.v.x, b.v.y, b.v.z, b.v.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint64_t word = b.word0 + j;
      // inside the segment (block -1 wraps below word_offset and fails the test)
      if (word - sg.word_offset < sg.n_words && lane < 31) word_off[word] = off;
      off += (wv[j >> 2] >> (8 * (j & 3))) & 0xffu;
    }
  }
}

}  // namespace

cudaError_t launch_index(const IndexParams &p, cudaStream_t stream) {
  const uint64_t n_chunks = p.chunk_end - p.chunk_begin;
  const uint32_t n_segs = p.seg_end - p.seg_begin;
  if (n_segs == 0) return cudaSuccess;
  // persistent warps over the chunks: at most one chunk per warp, at most p.grid CTAs of 8 warps
  const uint64_t want = (n_chunks + 7) / 8;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(p.grid ? p.grid : 1024u, want));
  if (n_chunks > 0) k_chunk_count<<<grid, 256, 0, stream>>>(p);
  const uint64_t warps_threads = (uint64_t)n_segs * 32;
  k_segment_scan<<<(unsigned)((warps_threads + 255) / 256), 256, 0, stream>>>(p);
  if (n_chunks > 0) k_tile_index<<<grid, 256, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace fptc

namespace fptc {
cudaError_t launch_word_offsets(const IndexParams &p, uint32_t *word_off, cudaStream_t stream) {
  const uint64_t n_chunks = p.chunk_end - p.chunk_begin;
  if (n_chunks == 0 || p.seg_end <= p.seg_begin) return cudaSuccess;
  const uint64_t want = (n_chunks + 7) / 8;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(p.grid ? p.grid : 1024u, want));
  k_word_offsets<<<grid, 256, 0, stream>>>(p, word_off);
  return cudaGetLastError();
}
}  // namespace fptc
