// Internal layout shared by the host plan and the CUDA kernels of libfptc.
// Nothing here is part of the C ABI.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

#include "fptc.h"

namespace fptc {

// Index work unit: a segment's symlen bytes are cut into chunks of 31 aligned
// 16-byte blocks (496 words, fewer in the segment's first and last chunk); the
// symbol offsets of the SymLen words (Sec. 4.2.1) are an exclusive scan over
// chunks, then over words inside a chunk.
constexpr uint32_t kChunkWords = 496;
// Chunks of a segment of n words for any placement of its first byte.
__host__ __device__ constexpr uint64_t chunks_of(uint64_t n) { return n ? ((n + 15) / 16 + 1 + 30) / 31 : 0; }
constexpr uint32_t kMaxLmax = 16;
constexpr uint32_t kChunkBad = 0xFFFFFFFFu;  // chunk sum sentinel: a symlen > 64 was seen

// Device status flags (mirror FPTC_FLAG_* in fptc.h).
constexpr unsigned int kFlagSymlenRange = 1u;
constexpr unsigned int kFlagBitOverrun = 2u;
constexpr unsigned int kFlagInvalidCode = 4u;
constexpr unsigned int kFlagSymbolCount = 8u;
constexpr unsigned int kFlagTimeout = 16u;

// Per-domain tables in device memory (copied to shared memory by the kernels).
struct DomainDev {
  uint32_t N, E, B1, B2;
  uint32_t lmax;
  uint32_t tile_windows;   // windows per tile
  uint32_t lut_offset;     // first entry of this domain's decode table
  uint32_t basis_offset;   // first float of this domain's E x N inverse-transform basis
  float scale[3];          // the plan's A_0, A_1, A_2 rounded to float
  uint32_t complete;       // 1 if the code lengths meet Kraft with equality (no invalid prefix)
  float unit[2][256];      // reconstruction at A_z = 1 for zones 0 and 1 (FP64 -> FP32)
};

// Entry B[k][n] of the inverse-transform basis of Eq. 1 (window size N):
// 1/2 for k = 0, else cos(pi (2n + 1) k / (2N)), evaluated in FP64 and rounded
// to FP32.  Host and device code evaluate the same expression.
__host__ __device__ inline float basis_value(uint32_t N, uint32_t n, uint32_t k) {
  return k == 0 ? 0.5f
                : static_cast<float>(cos(3.14159265358979323846 * (2.0 * n + 1.0) * k / (2.0 * N)));
}

// Host: the per-domain record of the decode kernels from a validated domain
// (shape, scales, whether the code is complete, reconstruction at A_z = 1 of
// Sec. 3.2); lut_offset, basis_offset and tile_windows are left 0.
void fill_domain_dev(const fptc_domain &dm, DomainDev *dd);

// The host encoder's FP64 level map of zone 0 or 1 (Eq. 2, Eq. 3) as its
// boundaries: bounds[L - 1], L = 1 .. 255, is the smallest double c whose
// level is L or more (-inf when every double's is, NaN when none is), so the
// level of any non-NaN c is the number of bounds <= c (the map is monotone in
// c, and a NaN bound is never <= c).
void host_zone_bounds(const fptc_domain &d, uint32_t zone, double *bounds);

// One segment, in tile-queue order (segments sorted by domain).
struct SegDev {
  uint64_t word_offset;
  uint64_t n_words;
  uint64_t n_samples;
  uint64_t out_offset;
  uint64_t level_offset;
  uint64_t n_windows;
  uint64_t tile_base;    // global index of the segment's first tile
  uint64_t n_tiles;
  uint64_t chunk_base;   // global index of the segment's first index chunk
  uint32_t n_chunks;
  uint32_t domain;
  uint32_t caller_index; // position in the caller's segment array
  uint32_t out_aligned;  // bit 0: out_offset % 4 == 0 (16-byte stores), bit 1: % 8 (32-byte), bit 2: % 32 (128-byte rows)
};

// Start of a tile in the SymLen stream: the word holding the tile's first symbol
// and how many earlier symbols of that word belong to the previous tile.
struct TileRec {
  uint64_t first_word;
  uint32_t skip;
  uint32_t pad;
};

struct DevStatus {
  unsigned int flags;
  unsigned int pad;
  unsigned long long first_bad;  // smallest caller index of a bad segment
};

struct IndexParams {
  const uint8_t *symlen;
  const SegDev *segs;
  const DomainDev *domains;
  uint32_t *chunk_sum;
  uint64_t *chunk_off;
  uint32_t *seg_bad;
  TileRec *tiles;
  DevStatus *status;
  uint64_t chunk_begin, chunk_end;  // chunk range of this launch
  uint32_t seg_begin, seg_end;      // segment range of this launch
  uint32_t grid;                    // CTAs of the chunk kernels (0: a default)
  uint32_t records;                 // 1: write a TileRec per tile (the kernels that read one)
};

struct DecodeParams {
  const uint64_t *words;
  const uint8_t *symlen;
  float *out;
  uint8_t *levels;          // optional level output
  const float *scale;       // optional run-time A_z [n_domains * 3]
  const SegDev *segs;
  const DomainDev *domains;
  const uint16_t *luts;
  const float *basis;
  const TileRec *tiles;
  const uint64_t *chunk_off;      // index chunk offsets (the warp-tile kernels locate their first tile)
  const uint32_t *seg_bad;
  DevStatus *status;
  uint64_t tile_begin, tile_end;  // tile range of this launch
  uint32_t seg_begin, seg_end;    // segment range covering it
  uint32_t lut_cap;               // decode-table entries that fit the shared buffer
  uint32_t coef_cap;              // tile_windows * E capacity of the shared tile buffers
};

// Shared-memory layout of the warp-tile kernel (decode_warp.cu).
constexpr uint32_t kWarpMaxDomains = 8;
struct WarpParams {
  uint32_t n_domains;
  uint32_t warp_off;    // first byte of the per-warp buffers
  uint32_t warp_bytes;  // bytes per warp
  uint32_t out_tma;     // 1: the output tensor map is valid (TMA stores for 128-byte aligned segments)
  uint32_t lut_off[kWarpMaxDomains];  // bytes
  uint32_t tab_off[kWarpMaxDomains];  // bytes
};

// Shared-memory layout of the tensor-core kernel (decode_tc.cu), bytes; the
// tables and per-warp buffers are laid out as for the warp-tile kernel.
struct TcParams {
  uint32_t a_off;      // per-warpgroup A operands (two buffers of a_buf bytes each)
  uint32_t a_buf;
  uint32_t b_off;      // B operand(s)
  uint32_t misc_off;   // mbarriers [warpgroups][2], tensor-memory address
  uint32_t tiles_off;  // output staging tiles start at the next 1024-byte boundary
  uint32_t pad[3];
};

struct BackwardParams {
  DecodeParams d;              // levels/words source, segments, tables
  const uint8_t *levels_in;    // saved levels, or null: decode again
  const float *grad_out;
  float *grad_coeffs;          // optional
  double *grad_scale;          // [n_domains * 3], zeroed by the host call
  uint32_t gx_cap;             // largest tile_windows * N of the plan
  uint32_t basis_cap;          // largest N * E of the plan
};

// Launch wrappers (index.cu, decode.cu, backward.cu).
cudaError_t launch_index(const IndexParams &p, cudaStream_t stream);
// per-word symbol offsets (index.cu) and the lossless / lossy kernels (decode_paper.cu) of the
// three-kernel schedule
cudaError_t launch_word_offsets(const IndexParams &p, uint32_t *word_off, cudaStream_t stream);
// halves: bit 0 runs the lossless kernel, bit 1 the lossy kernel.
cudaError_t launch_three_kernel(const DecodeParams &p, const uint32_t *word_off, uint8_t *levels,
                                uint64_t chunk_begin, uint64_t chunk_end, uint32_t halves, cudaStream_t stream);
// generic kernel (any N, E)
cudaError_t launch_decode(const DecodeParams &p, int kind, uint32_t threads, uint32_t grid, size_t smem,
                          cudaStream_t stream);
cudaError_t decode_smem_config(int kind, uint32_t threads, size_t smem);
cudaError_t decode_occupancy(int kind, uint32_t threads, size_t smem, int *ctas_per_sm);
size_t decode_smem_bytes(int kind, uint32_t threads, uint32_t lut_cap, uint32_t coef_cap);

// pipelined kernel for N = 32, E = 16 (decode_fixed.cu)
cudaError_t launch_fixed(const DecodeParams &p, uint32_t threads, uint32_t grid, size_t smem, cudaStream_t stream);
cudaError_t fixed_smem_config(uint32_t threads, size_t smem);
cudaError_t fixed_occupancy(uint32_t threads, size_t smem, int *ctas_per_sm);
size_t fixed_smem_bytes(uint32_t threads, uint32_t lut_cap, uint32_t coef_cap);

// warp-tile kernel for N = 32, E = 16 (decode_warp.cu); tiles of warp_tile_windows() windows
uint32_t warp_tile_windows();
size_t warp_smem_layout(uint32_t threads, const uint32_t *lmax, uint32_t n_domains, WarpParams *wp);
cudaError_t warp_smem_config(uint32_t threads, size_t smem);
cudaError_t warp_occupancy(uint32_t threads, size_t smem, int *ctas_per_sm);
cudaError_t launch_warp(const DecodeParams &p, const WarpParams &wp, const CUtensorMap &out_map, uint32_t threads,
                        uint32_t grid, size_t smem, cudaStream_t stream);
// Tensor map of an output buffer of `extent` floats viewed as rows of 32 floats
// (boxes of 32 x 32, 128-byte swizzle); false if it cannot be made.
bool encode_out_map(CUtensorMap *map, float *out, uint64_t extent);

// tensor-core kernel for N = 32, E = 16 (decode_tc.cu); mode = fptc_idct (not FP32)
uint32_t tc_tile_windows();
size_t tc_smem_layout(uint32_t mode, uint32_t threads, const uint32_t *lmax, uint32_t n_domains, WarpParams *wp,
                      TcParams *tp);
cudaError_t tc_smem_config(uint32_t mode, uint32_t threads, size_t smem);
cudaError_t tc_occupancy(uint32_t mode, uint32_t threads, size_t smem, int *ctas_per_sm);
cudaError_t tc_attributes(uint32_t mode, uint32_t threads, cudaFuncAttributes *attr);
cudaError_t launch_tc(const DecodeParams &p, const WarpParams &wp, const TcParams &tp, const CUtensorMap &out_map,
                      uint32_t mode, uint32_t threads, uint32_t grid, size_t smem, cudaStream_t stream);
// The tensor-core transform for shapes with E >= 32 (decode_tcs.cu): every domain the same
// (N, E) in {(32, 32), (64, 32), (128, 32), (128, 64)}; tiles of kTS / E windows; threads
// fixed per form and shape (tensor memory).
bool tcs_supported(uint32_t N, uint32_t E);
uint32_t tcs_tile_windows(uint32_t E);
uint32_t tcs_threads(uint32_t mode, uint32_t N, uint32_t E);
size_t tcs_smem_layout(uint32_t mode, uint32_t N, uint32_t E, const uint32_t *lmax, uint32_t n_domains,
                       WarpParams *wp, TcParams *tp);
cudaError_t tcs_smem_config(uint32_t mode, uint32_t N, uint32_t E, size_t smem);
cudaError_t tcs_occupancy(uint32_t mode, uint32_t N, uint32_t E, size_t smem, int *ctas_per_sm);
bool encode_out_map3(CUtensorMap *map, float *out, uint64_t extent, uint32_t N);
cudaError_t launch_tcs(const DecodeParams &p, const WarpParams &wp, const TcParams &tp, const CUtensorMap &out_map,
                       uint32_t mode, uint32_t N, uint32_t E, uint32_t grid, size_t smem, cudaStream_t stream);

// warp-tile kernel for other shapes: N in [4, 128] for every domain (several N
// in one plan), any E <= N (decode_shape.cu); tiles of shape_windows_per_tile(N,
// E) windows; `any`: some domain's N is not a power of two (shape_pow2_only
// false), served by the kernel instance that holds that transform
bool shape_supported(uint32_t N);
bool shape_pow2_only(uint32_t N);
uint32_t shape_windows_per_tile(uint32_t N, uint32_t E);
size_t shape_smem_layout(uint32_t threads, const uint32_t *lmax, const uint32_t *N, const uint32_t *E,
                         uint32_t n_domains, WarpParams *wp);
cudaError_t shape_smem_config(uint32_t threads, bool any, size_t smem);
cudaError_t shape_occupancy(uint32_t threads, bool any, size_t smem, int *ctas_per_sm);
cudaError_t launch_shape(const DecodeParams &p, const WarpParams &wp, const CUtensorMap &out_map, uint32_t threads,
                         bool any, uint32_t grid, size_t smem, cudaStream_t stream);

// adjoint for N = 32, E = 16 plans on the warp-tile machinery (backward_warp.cu)
size_t backward_warp_smem_layout(uint32_t threads, const uint32_t *lmax, uint32_t n_domains, WarpParams *wp);
cudaError_t backward_warp_smem_config(uint32_t threads, size_t smem);
cudaError_t launch_backward_warp(const BackwardParams &p, const WarpParams &wp, const CUtensorMap &gx_map,
                                 uint32_t threads, uint32_t grid, size_t smem, cudaStream_t stream);

cudaError_t launch_backward(const BackwardParams &p, uint32_t threads, uint32_t grid, size_t smem,
                            cudaStream_t stream);
size_t backward_smem_bytes(uint32_t threads, uint32_t lut_cap, uint32_t coef_cap, uint32_t gx_cap,
                           uint32_t basis_cap);
cudaError_t backward_smem_config(uint32_t threads, size_t smem);
cudaError_t backward_occupancy(uint32_t threads, size_t smem, int *ctas_per_sm);

}  // namespace fptc
