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
// table is read), with the next chunks' blocks loaded while the current ones
// are reduced; the chunk geometry is that of symlen_chunks.cuh.  Kernel 3 runs
// only for the kernels that read a record per tile: the warp-tile kernels
// locate the first tile of their range from the chunk offsets
// (symbol_word) and every later one from the tile decoded before it.
#include "symlen_chunks.cuh"

namespace fptc {
namespace {

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

// This warp's chunk range [c0, c1) of the launch.
__device__ __forceinline__ void warp_chunks(const IndexParams &p, uint64_t &c0, uint64_t &c1) {
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t n = p.chunk_end - p.chunk_begin;
  c0 = p.chunk_begin + n * gw / nw;
  c1 = p.chunk_begin + n * (gw + 1) / nw;
}

// Chunks in flight per warp: the loads of the next group of chunks are issued
// before the current group is reduced (four for the chunk sums, two for the
// tile index, whose group holds more state).

// Symlen blocks of chunks c .. c + P - 1 (clipped to c1) with their segments;
// the segment cursor s advances monotonically.
template <int P>
struct ChunkGroup {
  uint4 v[P];
  uint32_t seg[P];
};
template <int P>
__device__ __forceinline__ void load_group(const IndexParams &p, uint64_t c, uint64_t c1, uint32_t lane, uint32_t &s,
                                           ChunkGroup<P> &g) {
#pragma unroll
  for (int i = 0; i < P; ++i) {
    g.v[i] = make_uint4(0u, 0u, 0u, 0u);
    g.seg[i] = s;
    if (c + i < c1) {
      while (c + i >= p.segs[s].chunk_base + p.segs[s].n_chunks) ++s;
      g.seg[i] = s;
      g.v[i] = load_block(p.symlen, p.segs[s], c + i - p.segs[s].chunk_base, lane).v;
    }
  }
}

__global__ void __launch_bounds__(256, 4) k_chunk_count(IndexParams p) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t c0, c1;
  warp_chunks(p, c0, c1);
  if (c0 >= c1) return;
  uint32_t s = chunk_segment(p.segs, p.seg_begin, p.seg_end, c0);
  constexpr int kPipe = 4;
  ChunkGroup<kPipe> cur;
  load_group(p, c0, c1, lane, s, cur);
  for (uint64_t c = c0; c < c1; c += kPipe) {
    ChunkGroup<kPipe> nxt;
    load_group(p, c + kPipe, c1, lane, s, nxt);
#pragma unroll
    for (int i = 0; i < kPipe; ++i) {
      if (c + i >= c1) break;
      const uint32_t sum = __reduce_add_sync(0xffffffffu, block_sum(cur.v[i]));
      const uint32_t bad = __reduce_or_sync(0xffffffffu, block_over64(cur.v[i]) ? 1u : 0u);
      if (lane == 0) p.chunk_sum[c + i] = bad ? kChunkBad : sum;
    }
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

__global__ void __launch_bounds__(256, 3) k_tile_index(IndexParams p) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t c0, c1;
  warp_chunks(p, c0, c1);
  if (c0 >= c1) return;
  uint32_t s = chunk_segment(p.segs, p.seg_begin, p.seg_end, c0);
  constexpr int kPipe = 2;
  ChunkGroup<kPipe> cur;
  load_group(p, c0, c1, lane, s, cur);
  uint64_t off_cur[kPipe];
#pragma unroll
  for (int i = 0; i < kPipe; ++i) off_cur[i] = c0 + i < c1 ? p.chunk_off[c0 + i] : 0;
  for (uint64_t c = c0; c < c1; c += kPipe) {
    ChunkGroup<kPipe> nxt;
    load_group(p, c + kPipe, c1, lane, s, nxt);
    uint64_t off_nxt[kPipe];
#pragma unroll
    for (int i = 0; i < kPipe; ++i) off_nxt[i] = c + kPipe + i < c1 ? p.chunk_off[c + kPipe + i] : 0;
#pragma unroll
    for (int i = 0; i < kPipe; ++i) {
      if (c + i >= c1) break;
      const uint32_t si = cur.seg[i];
      if (p.seg_bad[si] != 0) continue;  // uniform over the warp
      const SegDev &sg = p.segs[si];
      const DomainDev &dm = p.domains[sg.domain];
      const uint64_t te = (uint64_t)dm.tile_windows * dm.E;  // symbols per tile
      const uint4 bv = cur.v[i];
      const uint32_t tsum = block_sum(bv);
      uint32_t x = tsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
      }
      if (tsum == 0) continue;
      uint64_t off = off_cur[i] + (x - tsum);  // symbol offset (in the segment) of the block's first word
      // first tile whose start is >= off
      uint64_t tn = off < 0xFFFFFFFFull && te < 0xFFFFFFFFull ? ((uint32_t)off + (uint32_t)te - 1u) / (uint32_t)te
                                                                : (off + te - 1) / te;
      uint64_t ns = tn * te;
      if (ns >= off + tsum) continue;  // most blocks hold no tile start (a tile is thousands of symbols)
      const uint32_t wv[4] = {bv.x, bv.y, bv.z, bv.w};
      // global word index of byte 0 of this lane's block (as load_block computes it)
      const uintptr_t a0 = reinterpret_cast<uintptr_t>(p.symlen + sg.word_offset);
      const uint64_t word0 = sg.word_offset + (uint64_t)(((a0 + 15) & ~uintptr_t(15)) +
                                                         16 * (uintptr_t)(31 * (c + i - sg.chunk_base) + lane) - 16 - a0);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uint64_t end = off + ((wv[j >> 2] >> (8 * (j & 3))) & 0xffu);
        while (ns < end) {
          if (tn < sg.n_tiles) {
            TileRec r;
            r.first_word = word0 + j;
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
    cur = nxt;
#pragma unroll
    for (int i = 0; i < kPipe; ++i) off_cur[i] = off_nxt[i];
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
  if (n_chunks > 0 && p.records) k_tile_index<<<grid, 256, 0, stream>>>(p);
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
