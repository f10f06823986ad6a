// The decoder as the paper lays it out on the GPU (Sec. 4.2), kept as an
// in-library comparison for the fused persistent kernels (plan schedule
// FPTC_SCHEDULE_THREE_KERNEL):
//   1. a prefix sum over symlen gives every word the position of its first
//      symbol (k_chunk_count, k_segment_scan, k_word_offsets in index.cu);
//   2. the lossless kernel: one thread per word decodes its symlen[w] codewords
//      with the decode table and writes the levels to a dense global byte array;
//   3. the lossy kernel: one thread per output sample reads the E levels of its
//      window, dequantizes them and sums the inverse DCT for its sample.
// Every intermediate goes through global memory (the level array is written
// once and read by all N threads of its window), which is what the fused
// kernels avoid.
#include "device_util.cuh"

namespace fptc {
namespace {

constexpr uint32_t kLosslessThreads = 512;  // one chunk (31 blocks of 16 words) per CTA
constexpr uint32_t kLossyThreads = 256;

__device__ __forceinline__ uint32_t segment_of_chunk(const SegDev *segs, uint32_t lo, uint32_t hi, uint64_t c) {
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (segs[mid].chunk_base <= c)
      lo = mid;
    else
      hi = mid;
  }
  while (c >= segs[lo].chunk_base + segs[lo].n_chunks) ++lo;
  return lo;
}

__global__ void __launch_bounds__(kLosslessThreads) k_lossless(const DecodeParams p, const uint32_t *word_off,
                                                               uint8_t *levels, uint64_t chunk_begin) {
  __shared__ uint32_t s_seg;
  const uint64_t c = chunk_begin + blockIdx.x;
  if (threadIdx.x == 0) s_seg = segment_of_chunk(p.segs, p.seg_begin, p.seg_end, c);
  __syncthreads();
  const uint32_t s = s_seg;
  const SegDev &sg = p.segs[s];
  if (p.seg_bad[s] != 0 || threadIdx.x >= 31 * 16) return;
  // word of this thread: byte threadIdx.x % 16 of block 31 k - 1 + threadIdx.x / 16 (the index's chunk geometry)
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(p.symlen + sg.word_offset);
  const uintptr_t blk = ((a0 + 15) & ~uintptr_t(15)) + 16 * (uintptr_t)(31 * (c - sg.chunk_base) + threadIdx.x / 16) - 16;
  const uintptr_t a = blk + (threadIdx.x & 15u);
  if (a < a0 || a >= a0 + sg.n_words) return;
  const uint64_t wi = sg.word_offset + (uint64_t)(a - a0);
  const DomainDev &dm = p.domains[sg.domain];
  const uint16_t *lut = p.luts + dm.lut_offset;
  const uint32_t shift = 64u - dm.lmax;
  const uint32_t n = __ldg(p.symlen + wi);
  uint64_t w = __ldg(p.words + wi);
  const uint64_t total = sg.n_windows * dm.E;
  uint64_t q = word_off[wi];
  uint8_t *dst = levels + sg.level_offset;
  uint32_t used = 0;
  unsigned err = 0;
  for (uint32_t j = 0; j < n; ++j, ++q) {
    const uint32_t e = __ldg(lut + (uint32_t)(w >> shift));
    const uint32_t len = e >> 8;
    if (len == 0) {
      err |= kFlagInvalidCode;
      break;
    }
    used += len;
    if (used > 64u) {
      err |= kFlagBitOverrun;
      break;
    }
    w <<= len;
    if (q < total) dst[q] = (uint8_t)(e & 0xffu);
  }
  if (err) flag_bad(p.status, err, sg.caller_index);
}

__global__ void __launch_bounds__(kLossyThreads) k_lossy(const DecodeParams p, const uint8_t *levels) {
  __shared__ uint32_t s_seg;
  const uint64_t g = p.tile_begin + blockIdx.x;
  if (threadIdx.x == 0) s_seg = find_segment(p.segs, p.seg_begin, p.seg_end, g);
  __syncthreads();
  uint32_t s = s_seg;
  while (g >= p.segs[s].tile_base + p.segs[s].n_tiles) ++s;
  const SegDev &sg = p.segs[s];
  if (p.seg_bad[s] != 0) return;
  const DomainDev &dm = p.domains[sg.domain];
  const uint32_t N = dm.N, E = dm.E, B1 = dm.B1, B2 = dm.B2;
  const float a0 = p.scale ? p.scale[sg.domain * 3 + 0] : dm.scale[0];
  const float a1 = p.scale ? p.scale[sg.domain * 3 + 1] : dm.scale[1];
  const float A0 = a0 > 1e-30f ? a0 : 0.0f, A1 = a1 > 1e-30f ? a1 : 0.0f;
  const float *basis = p.basis + dm.basis_offset;
  const uint64_t s_begin = (g - sg.tile_base) * dm.tile_windows * N;
  const uint64_t s_lim = s_begin + (uint64_t)dm.tile_windows * N;
  const uint64_t s_end = s_lim < sg.n_samples ? s_lim : sg.n_samples;
  const uint8_t *lev = levels + sg.level_offset;
  float *out = p.out + sg.out_offset;
  for (uint64_t i = s_begin + threadIdx.x; i < s_end; i += kLossyThreads) {
    const uint64_t win = i / N;
    const uint32_t n = (uint32_t)(i - win * N);
    float x = 0.0f;
    for (uint32_t k = 0; k < E; ++k) {
      const uint32_t L = __ldg(lev + win * E + k);
      const uint32_t z = k < B1 ? 0u : (k < B2 ? 1u : 2u);
      const float c = z == 0 ? A0 * __ldg(&dm.unit[0][L]) : (z == 1 ? A1 * __ldg(&dm.unit[1][L]) : 0.0f);
      x = fmaf(c, __ldg(basis + k * N + n), x);
    }
    out[i] = x;
  }
}

}  // namespace

cudaError_t launch_three_kernel(const DecodeParams &p, const uint32_t *word_off, uint8_t *levels,
                                uint64_t chunk_begin, uint64_t chunk_end, uint32_t halves, cudaStream_t stream) {
  if ((halves & 1u) && chunk_end > chunk_begin) {
    if (chunk_end - chunk_begin > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    k_lossless<<<(unsigned)(chunk_end - chunk_begin), kLosslessThreads, 0, stream>>>(p, word_off, levels, chunk_begin);
  }
  if ((halves & 2u) && p.tile_end > p.tile_begin) {
    if (p.tile_end - p.tile_begin > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    k_lossy<<<(unsigned)(p.tile_end - p.tile_begin), kLossyThreads, 0, stream>>>(p, levels);
  }
  return cudaGetLastError();
}

}  // namespace fptc
