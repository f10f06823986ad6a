// fptc_decode_stream_noalloc: decode one compressed stream without allocating.
//
// Some callers cannot allocate device memory at the time they decode: code that
// runs inside a framework's memory pool or an allocator callback (where a
// cudaMalloc would re-enter the allocator or break its accounting), real-time
// or embedded-serving paths that forbid any allocation after start-up, and
// processes whose device memory is fully reserved by another runtime.  For them
// this entry point runs the same SymLen index kernels and the same generic
// decode kernel as a plan, but every piece of working memory (the domain
// tables, the segment/chunk/tile records, the index scratch and the status
// word) lives in one file-scope device array of fixed size.  The caller still
// passes the input words/symlen and the output buffer.
#include <algorithm>
#include <cstring>

#include "fptc.h"
#include "fptc_codec.h"
#include "fptc_internal.h"
#include "host_util.h"

namespace fptc {
namespace {

// Limits of the allocation-free path (see fptc.h).
constexpr uint64_t kNaMaxSamples = 1ull << 26;                   // 67,108,864 samples per call
constexpr uint32_t kNaTileSamples = 4096;                        // generic kernel tile size
constexpr uint64_t kNaMaxWords = kNaMaxSamples;                  // words <= symbols <= samples (E <= N)
constexpr uint64_t kNaMaxChunks = chunks_of(kNaMaxWords);
constexpr uint32_t kNaMaxLmax = 12;                              // decode table of 4096 entries

// Byte layout of the scratch array (each piece 256-byte aligned).
constexpr size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffStatus = 0;
constexpr size_t kOffSegBad = a256(kOffStatus + sizeof(DevStatus));
constexpr size_t kOffSeg = a256(kOffSegBad + sizeof(uint32_t));
constexpr size_t kOffDom = a256(kOffSeg + sizeof(SegDev));
constexpr size_t kOffLut = a256(kOffDom + sizeof(DomainDev));
constexpr size_t kOffBasis = a256(kOffLut + (size_t(2) << kNaMaxLmax));
constexpr size_t kOffChunkSum = a256(kOffBasis + 128 * 128 * sizeof(float));
constexpr size_t kOffChunkOff = a256(kOffChunkSum + kNaMaxChunks * sizeof(uint32_t));
constexpr size_t kOffTiles = a256(kOffChunkOff + kNaMaxChunks * sizeof(uint64_t));
// a tile holds floor(4096 / N) windows, i.e. >= 4096 - N + 1 >= 3969 samples (N <= 128)
constexpr uint64_t kNaTileCap = kNaMaxSamples / 3968 + 2;
constexpr size_t kScratchBytes = a256(kOffTiles + kNaTileCap * sizeof(TileRec));

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Everything the decode needs besides the caller's buffers, passed by value as
// the set-up kernel's argument (about 10 KB): no host memory is read once the
// launch returns, and no host-to-device copy is made.
struct NaSetup {
  DevStatus status;                 // cleared status word
  SegDev seg;
  DomainDev dom;
  uint32_t lut_entries;
  uint16_t lut[1u << kNaMaxLmax];
};
static_assert(sizeof(NaSetup) <= 32000, "kernel arguments are limited to 32,764 bytes");

// Fills the scratch array: status word, segment flag, records, decode table and
// the E x N inverse-transform basis (the same expression the plan evaluates on
// the host).  Device code names the array directly.
__global__ void k_na_setup(const __grid_constant__ NaSetup a) {
  unsigned char *const scr = g_scratch;
  if (threadIdx.x == 0) {
    *reinterpret_cast<DevStatus *>(scr + kOffStatus) = a.status;
    *reinterpret_cast<uint32_t *>(scr + kOffSegBad) = 0u;
    *reinterpret_cast<SegDev *>(scr + kOffSeg) = a.seg;
    *reinterpret_cast<DomainDev *>(scr + kOffDom) = a.dom;
  }
  uint16_t *const lut = reinterpret_cast<uint16_t *>(scr + kOffLut);
  for (uint32_t i = threadIdx.x; i < a.lut_entries; i += blockDim.x) lut[i] = a.lut[i];
  float *const basis = reinterpret_cast<float *>(scr + kOffBasis);
  const uint32_t N = a.dom.N, E = a.dom.E;
  for (uint32_t i = threadIdx.x; i < N * E; i += blockDim.x) basis[i] = basis_value(N, i % N, i / N);
}

// Device address of g_scratch on the current device.  Host code may not use
// the symbol itself (it names a host-side stand-in).  Looked up on every call:
// after the library's device code is loaded this is a table lookup, and a
// fresh lookup stays right after the context has been reset.
fptc_status scratch_for_current_device(unsigned char **out) {
  void *ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess || !ptr) {
    set_error("cudaGetSymbolAddress of the decode scratch failed: %s", cudaGetErrorString(e));
    return FPTC_ERR_CUDA;
  }
  *out = static_cast<unsigned char *>(ptr);
  return FPTC_OK;
}

}  // namespace
}  // namespace fptc

using namespace fptc;

extern "C" fptc_status fptc_decode_stream_noalloc(const fptc_domain *domain, const uint64_t *d_words,
                                                  const uint8_t *d_symlen, uint64_t n_words, uint64_t n_samples,
                                                  float *d_out, fptc_stream stream) {
  clear_error();
  fptc_status st = fptc_validate_domain(domain);
  if (st != FPTC_OK) return st;
  const fptc_domain &dm = *domain;
  if (dm.lmax > kNaMaxLmax) {
    set_error("the allocation-free decode supports lmax <= %u (got %u)", kNaMaxLmax, dm.lmax);
    return FPTC_ERR_UNSUPPORTED;
  }
  if (n_samples > kNaMaxSamples) {
    set_error("the allocation-free decode takes at most %llu samples per call (got %llu)",
              (unsigned long long)kNaMaxSamples, (unsigned long long)n_samples);
    return FPTC_ERR_UNSUPPORTED;
  }
  const uint64_t W = (n_samples + dm.N - 1) / dm.N;
  const uint64_t L = W * dm.E;
  if (n_words < (L + 63) / 64 || n_words > L) {
    set_error("%llu words cannot hold %llu symbols", (unsigned long long)n_words, (unsigned long long)L);
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  if (n_samples == 0) return FPTC_OK;
  if (!d_words || !d_symlen || !d_out || (reinterpret_cast<uintptr_t>(d_words) & 7u) ||
      (reinterpret_cast<uintptr_t>(d_out) & 3u)) {
    set_error("d_words (8-byte aligned), d_symlen and d_out (4-byte aligned) are required");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("cudaGetDevice: %s", cudaGetErrorString(e));
    return FPTC_ERR_CUDA;
  }
  unsigned char *scr = nullptr;
  if ((st = scratch_for_current_device(&scr)) != FPTC_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // ---- records and tables, built on the host in the set-up kernel's argument
  // (a stack object: no heap allocation)
  NaSetup a;
  std::memset(&a, 0, sizeof(a));
  a.status = DevStatus{0u, 0u, ~0ull};
  DomainDev &dd = a.dom;
  fill_domain_dev(dm, &dd);  // the plan's own per-domain record
  dd.tile_windows = std::max<uint32_t>(1u, kNaTileSamples / dm.N);
  dd.lut_offset = 0;
  dd.basis_offset = 0;
  a.lut_entries = 1u << dm.lmax;
  if ((st = fptc_build_decode_table(&dm, a.lut)) != FPTC_OK) return st;
  SegDev &sg = a.seg;
  sg.word_offset = 0;
  sg.n_words = n_words;
  sg.n_samples = n_samples;
  sg.out_offset = 0;
  sg.level_offset = 0;
  sg.n_windows = W;
  sg.tile_base = 0;
  sg.n_tiles = (W + dd.tile_windows - 1) / dd.tile_windows;
  sg.chunk_base = 0;
  sg.n_chunks = (uint32_t)chunks_of(n_words);
  sg.domain = 0;
  sg.caller_index = 0;
  sg.out_aligned = (reinterpret_cast<uintptr_t>(d_out) & 15u) == 0;
  if (sg.n_tiles > kNaTileCap) {
    set_error("too many tiles for the allocation-free decode");
    return FPTC_ERR_UNSUPPORTED;
  }

  // ---- set-up kernel: the scratch array's records, tables and cleared status
  {
    void *args[] = {&a};
    e = cudaLaunchKernel(reinterpret_cast<const void *>(&k_na_setup), dim3(1), dim3(256), args, 0, s);
  }
  if (e != cudaSuccess) {
    set_error("allocation-free decode set-up launch: %s", cudaGetErrorString(e));
    return FPTC_ERR_CUDA;
  }

  // ---- index + generic decode kernel on the scratch
  IndexParams ip{};
  ip.symlen = d_symlen;
  ip.segs = reinterpret_cast<const SegDev *>(scr + kOffSeg);
  ip.domains = reinterpret_cast<const DomainDev *>(scr + kOffDom);
  ip.chunk_sum = reinterpret_cast<uint32_t *>(scr + kOffChunkSum);
  ip.chunk_off = reinterpret_cast<uint64_t *>(scr + kOffChunkOff);
  ip.seg_bad = reinterpret_cast<uint32_t *>(scr + kOffSegBad);
  ip.tiles = reinterpret_cast<TileRec *>(scr + kOffTiles);
  ip.status = reinterpret_cast<DevStatus *>(scr + kOffStatus);
  ip.chunk_begin = 0;
  ip.chunk_end = sg.n_chunks;
  ip.seg_begin = 0;
  ip.seg_end = 1;
  ip.grid = 0;
  ip.records = 1;
  e = launch_index(ip, s);
  if (e != cudaSuccess) {
    set_error("allocation-free index launch: %s", cudaGetErrorString(e));
    return FPTC_ERR_CUDA;
  }
  DecodeParams dp{};
  dp.words = d_words;
  dp.symlen = d_symlen;
  dp.out = d_out;
  dp.levels = nullptr;
  dp.scale = nullptr;
  dp.segs = ip.segs;
  dp.domains = ip.domains;
  dp.luts = reinterpret_cast<const uint16_t *>(scr + kOffLut);
  dp.basis = reinterpret_cast<const float *>(scr + kOffBasis);
  dp.tiles = ip.tiles;
  dp.chunk_off = ip.chunk_off;
  dp.seg_bad = ip.seg_bad;
  dp.status = ip.status;
  dp.tile_begin = 0;
  dp.tile_end = sg.n_tiles;
  dp.seg_begin = 0;
  dp.seg_end = 1;
  dp.lut_cap = 1u << dm.lmax;
  dp.coef_cap = dd.tile_windows * dm.E;
  const uint32_t threads = 256;
  const size_t smem = decode_smem_bytes(FPTC_KERNEL_GENERIC, threads, dp.lut_cap, dp.coef_cap);
  if ((e = decode_smem_config(FPTC_KERNEL_GENERIC, threads, smem)) == cudaSuccess) {
    int occ = 1, sms = 1;
    decode_occupancy(FPTC_KERNEL_GENERIC, threads, smem, &occ);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms * std::max(occ, 1),
                                                                              sg.n_tiles));
    e = launch_decode(dp, FPTC_KERNEL_GENERIC, threads, grid, smem, s);
  }
  if (e != cudaSuccess) {
    set_error("allocation-free decode launch: %s", cudaGetErrorString(e));
    return FPTC_ERR_CUDA;
  }
  return FPTC_OK;
}
