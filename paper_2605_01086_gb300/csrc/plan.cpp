// Host side of libfptc: plan creation (validation, decode tables,
// reconstruction tables, tile queue), the C ABI entry points and the launch
// sequences of the decoder (index kernels, then the fused decode kernel).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "fptc.h"
#include "fptc_codec.h"
#include "fptc_internal.h"
#include "host_util.h"

using namespace fptc;

struct fptc_plan {
  int device = 0;
  int sm_count = 0;
  fptc_plan_options opts{};
  std::vector<fptc_domain> domains;
  std::vector<fptc_segment> caller_segs;
  std::vector<uint32_t> queue;           // queue position -> caller index
  std::vector<SegDev> segs;              // queue order
  std::vector<DomainDev> dom_dev;
  std::vector<uint64_t> level_off;       // caller order
  uint64_t n_tiles = 0, n_chunks = 0, n_levels = 0;
  uint64_t words_extent = 0, out_extent = 0, n_samples = 0, n_words = 0;
  // device memory owned by the plan
  DomainDev *d_domains = nullptr;
  SegDev *d_segs = nullptr;
  uint16_t *d_luts = nullptr;
  float *d_basis = nullptr;
  uint32_t *d_chunk_sum = nullptr;
  uint64_t *d_chunk_off = nullptr;
  uint32_t *d_seg_bad = nullptr;
  uint32_t *d_word_off = nullptr;   // three-kernel schedule: symbol offset of every word
  uint8_t *d_lev_scratch = nullptr; // three-kernel schedule: the level array
  TileRec *d_tiles = nullptr;
  uint64_t tiles_capacity = 0;
  DevStatus *d_status = nullptr;
  size_t device_bytes = 0;
  // launch settings
  int kind = FPTC_KERNEL_GENERIC;   // fptc_kernel in use
  bool shape = false;     // every domain has N in [4, 128] and the warp-tile kernel of
                          // decode_shape.cu serves the plan (N = 32, E = 16 plans use decode_warp.cu)
  uint32_t tcs_N = 0, tcs_E = 0;  // the tensor-core kernel of decode_tcs.cu serves this shape (0: decode_tc.cu)
  bool shape_any = false; // a domain's N is not a power of two (the shape kernel instance with that transform)
  WarpParams wp{};
  TcParams tp{};
  uint32_t threads = 256, grid = 0, ctas_per_sm = 0;
  size_t smem = 0;
  uint32_t lut_cap = 0, coef_cap = 0, gx_cap = 0, basis_cap = 0;
  uint32_t b_threads = 256, b_grid = 0;
  size_t b_smem = 0;
  bool b_warp = false;    // backward on the warp-tile adjoint kernel
  WarpParams b_wp{};
  static constexpr int kAux = 4;        // copy-back streams of the end-to-end decode
  static constexpr int kPieces = 16;    // decode pieces of the end-to-end decode
  cudaStream_t aux[kAux] = {};
  cudaStream_t up = nullptr;            // upload stream of the end-to-end decode
  cudaEvent_t ev[kPieces] = {};         // piece k decoded
  cudaEvent_t evh[kPieces] = {};        // piece k's words uploaded
  cudaEvent_t ev_start = nullptr;       // the caller's stream reached the end-to-end decode
};

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

fptc_status cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FPTC_ERR_OUT_OF_MEMORY : FPTC_ERR_CUDA;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src, size_t *bytes) {
  const size_t n = std::max<size_t>(src.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), n);
  if (e != cudaSuccess) return e;
  *bytes += n;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

void free_device(fptc_plan *p);

// Frees a plan and the device memory, streams and events it holds, on its
// device (a plan that never reached the device holds none).
struct PlanDeleter {
  void operator()(fptc_plan *p) const;
};

void free_device(fptc_plan *p) {
  cudaFree(p->d_domains);
  cudaFree(p->d_segs);
  cudaFree(p->d_luts);
  cudaFree(p->d_basis);
  cudaFree(p->d_chunk_sum);
  cudaFree(p->d_chunk_off);
  cudaFree(p->d_seg_bad);
  cudaFree(p->d_word_off);
  cudaFree(p->d_lev_scratch);
  cudaFree(p->d_tiles);
  cudaFree(p->d_status);
  for (auto &a : p->aux)
    if (a) cudaStreamDestroy(a);
  if (p->up) cudaStreamDestroy(p->up);
  for (auto &e : p->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : p->evh)
    if (e) cudaEventDestroy(e);
  if (p->ev_start) cudaEventDestroy(p->ev_start);
}

void PlanDeleter::operator()(fptc_plan *p) const {
  if (!p) return;
  if (p->d_domains || p->d_segs || p->d_luts || p->d_basis || p->d_chunk_sum || p->d_chunk_off || p->d_seg_bad ||
      p->d_word_off || p->d_lev_scratch || p->d_tiles || p->d_status || p->up || p->ev_start || p->aux[0] ||
      p->ev[0] || p->evh[0]) {
    DeviceGuard g(p->device);
    free_device(p);
  }
  delete p;
}

// Reconstruction at A_z = 1 (the inverse zone maps of Sec. 3.2), FP64 then FP32.
void unit_tables(const fptc_domain &d, float unit[2][256]) {
  const double mu = d.mu, a = d.alpha1, span = 1.0 - d.alpha1;
  for (int L = 0; L < 256; ++L) {
    double u0 = 0.0, u1 = 0.0;
    if (L > 128) {
      u0 = (std::pow(1.0 + mu, (L - 128) / 127.0) - 1.0) / mu;
      u1 = a + (L - 129) / 126.0 * span;
    } else if (L < 128) {
      u0 = -(std::pow(1.0 + mu, (128 - L) / 128.0) - 1.0) / mu;
      u1 = -(a + (127 - L) / 127.0 * span);
    }
    unit[0][L] = static_cast<float>(u0);
    unit[1][L] = static_cast<float>(u1);
  }
}

}  // namespace

void fptc::fill_domain_dev(const fptc_domain &dm, DomainDev *dd) {
  std::memset(dd, 0, sizeof(*dd));
  dd->N = dm.N;
  dd->E = dm.E;
  dd->B1 = dm.B1;
  dd->B2 = dm.B2;
  dd->lmax = dm.lmax;
  for (int z = 0; z < 3; ++z) dd->scale[z] = static_cast<float>(dm.scale[z]);
  uint64_t kraft = 0;
  for (int sy = 0; sy < 256; ++sy)
    if (dm.code_len[sy]) kraft += uint64_t(1) << (dm.lmax - dm.code_len[sy]);
  dd->complete = kraft == (uint64_t(1) << dm.lmax);
  unit_tables(dm, dd->unit);
}

namespace {

// Layout of the tile queue for a tile size (target samples per tile).
void layout_tiles(fptc_plan *p, uint32_t tile_samples) {
  p->coef_cap = 0;
  p->gx_cap = 0;
  const bool shape = p->kind == FPTC_KERNEL_WARP_TILE && p->shape;
  for (auto &dd : p->dom_dev) {
    dd.tile_windows = shape ? shape_windows_per_tile(dd.N, dd.E) : std::max<uint32_t>(1u, tile_samples / dd.N);
    p->coef_cap = std::max(p->coef_cap, dd.tile_windows * dd.E);
    p->gx_cap = std::max(p->gx_cap, dd.tile_windows * dd.N);
  }
  uint64_t t = 0;
  for (auto &s : p->segs) {
    const uint32_t T = p->dom_dev[s.domain].tile_windows;
    s.tile_base = t;
    s.n_tiles = (s.n_windows + T - 1) / T;
    t += s.n_tiles;
  }
  p->n_tiles = t;
}

// FPTC_ERR_UNSUPPORTED with the sizes when a kernel's shared memory at `threads`
// exceeds what one CTA may opt in to on the current device.
fptc_status smem_fits(const char *kernel, uint32_t threads, size_t smem) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem <= (size_t)optin) return FPTC_OK;
  set_error("the %s kernel at %u threads needs %zu bytes of shared memory with these domains' tables; a CTA may "
            "use %d (fewer threads, or 0 to choose)",
            kernel, threads, smem, optin);
  return FPTC_ERR_UNSUPPORTED;
}

fptc_status configure_launch(fptc_plan *p) {
  uint32_t threads = p->opts.threads ? p->opts.threads : (p->kind == FPTC_KERNEL_TENSOR ? 512u : 256u);
  const bool shape = p->kind == FPTC_KERNEL_WARP_TILE && p->shape;
  std::vector<uint32_t> lm, ns, es;
  for (const auto &d : p->domains) {
    lm.push_back(d.lmax);
    ns.push_back(d.N);
    es.push_back(d.E);
  }
  if (p->kind == FPTC_KERNEL_WARP_TILE && p->opts.threads == 0) {
    // as many warps per SM as one CTA's shared memory allows (32 at most; 16
    // for other shapes, whose transform wants more registers per thread)
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    WarpParams probe{};
    threads = 128;
    if (shape) {
      for (uint32_t t : {512u, 256u})
        if (shape_smem_layout(t, lm.data(), ns.data(), es.data(), (uint32_t)lm.size(), &probe) <= (size_t)optin) {
          threads = t;
          break;
        }
    } else {
      // 896 before 1024: 28 warps run without spills (72 registers), 32 would spill at 64
      for (uint32_t t : {896u, 1024u, 768u, 512u, 256u})
        if (warp_smem_layout(t, lm.data(), (uint32_t)lm.size(), &probe) <= (size_t)optin) {
          threads = t;
          break;
        }
    }
  }
  if (p->kind == FPTC_KERNEL_TENSOR && p->tcs_N) threads = tcs_threads(p->opts.idct, p->tcs_N, p->tcs_E);
  const bool t_ok = (p->kind == FPTC_KERNEL_TENSOR && p->tcs_N) ? threads > 0
                    : shape ? (threads == 256 || threads == 512 || threads == 768)
                          : (threads == 128 || threads == 256 || threads == 512 ||
                             ((threads == 768 || threads == 896 || threads == 1024) &&
                              p->kind == FPTC_KERNEL_WARP_TILE) ||
                             ((threads == 384 || threads == 640 || threads == 768 || threads == 896) &&
                              p->kind == FPTC_KERNEL_TENSOR));
  if (!t_ok) {
    set_error("threads must be 128, 256 or 512 (768, 896 and 1024 also for the warp-tile kernel, 384, 640, 768 and "
              "896 for the tensor-core kernel; 256, 512 or 768 for the warp-tile kernel of other shapes; got %u)",
              threads);
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  p->threads = threads;
  cudaError_t e;
  int occ = 0;
  if (p->kind == FPTC_KERNEL_BLOCK_TILE) {
    p->smem = fixed_smem_bytes(threads, p->lut_cap, p->coef_cap);
    e = fixed_smem_config(threads, p->smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode shared-memory size");
    e = fixed_occupancy(threads, p->smem, &occ);
  } else if (p->kind == FPTC_KERNEL_TENSOR && p->tcs_N) {
    // the shape kernel: threads fixed by its form and shape (tensor memory), one CTA per SM
    p->smem = tcs_smem_layout(p->opts.idct, p->tcs_N, p->tcs_E, lm.data(), (uint32_t)lm.size(), &p->wp, &p->tp);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (p->smem > (size_t)optin) {
      set_error("tensor-core kernel of shape N = %u, E = %u does not fit shared memory", p->tcs_N, p->tcs_E);
      return FPTC_ERR_UNSUPPORTED;
    }
    e = tcs_smem_config(p->opts.idct, p->tcs_N, p->tcs_E, p->smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode shared-memory size");
    e = tcs_occupancy(p->opts.idct, p->tcs_N, p->tcs_E, p->smem, &occ);
    if (e == cudaSuccess) occ = std::min<int>(occ, 1);
  } else if (p->kind == FPTC_KERNEL_TENSOR) {
    if (p->opts.threads == 0) {
      // as many warpgroups as one CTA's shared memory and tensor memory allow (7 at most)
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      WarpParams pw{};
      TcParams pt{};
      threads = 128;
      for (uint32_t t : {896u, 768u, 640u, 512u, 384u, 256u})
        if (tc_smem_layout(p->opts.idct, t, lm.data(), (uint32_t)lm.size(), &pw, &pt) <= (size_t)optin) {
          threads = t;
          break;
        }
      p->threads = threads;
    }
    p->smem = tc_smem_layout(p->opts.idct, threads, lm.data(), (uint32_t)lm.size(), &p->wp, &p->tp);
    if (p->smem == ~size_t(0)) {
      set_error("the tensor-core kernel at %u threads (%u warpgroups) needs more than the 512 tensor-memory "
                "columns of an SM in this form (at most 640 threads for 3xTF32, 896 for the others)",
                threads, threads / 128);
      return FPTC_ERR_UNSUPPORTED;
    }
    if (const fptc_status fs = smem_fits("tensor-core", threads, p->smem); fs != FPTC_OK) return fs;
    e = tc_smem_config(p->opts.idct, threads, p->smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode shared-memory size");
    e = tc_occupancy(p->opts.idct, threads, p->smem, &occ);
    // one CTA per SM (tensor memory)
    if (std::getenv("FPTC_DEBUG")) {
      cudaFuncAttributes fa{};
      tc_attributes(p->opts.idct, threads, &fa);
      std::fprintf(stderr, "fptc: tensor kernel threads %u regs %d static smem %zu max dyn smem %d dyn %zu occupancy %d\n",
                   threads, fa.numRegs, fa.sharedSizeBytes, fa.maxDynamicSharedSizeBytes, p->smem, occ);
    }
    if (e == cudaSuccess) occ = std::min<int>(occ, 1);
  } else if (shape) {
    p->smem = shape_smem_layout(threads, lm.data(), ns.data(), es.data(), (uint32_t)lm.size(), &p->wp);
    if (const fptc_status fs = smem_fits("warp-tile", threads, p->smem); fs != FPTC_OK) return fs;
    e = shape_smem_config(threads, p->shape_any, p->smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode shared-memory size");
    e = shape_occupancy(threads, p->shape_any, p->smem, &occ);
  } else if (p->kind == FPTC_KERNEL_WARP_TILE) {
    p->smem = warp_smem_layout(threads, lm.data(), (uint32_t)lm.size(), &p->wp);
    if (const fptc_status fs = smem_fits("warp-tile", threads, p->smem); fs != FPTC_OK) return fs;
    e = warp_smem_config(threads, p->smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode shared-memory size");
    e = warp_occupancy(threads, p->smem, &occ);
  } else {
    p->smem = decode_smem_bytes(p->kind, threads, p->lut_cap, p->coef_cap);
    e = decode_smem_config(p->kind, threads, p->smem);
    if (e != cudaSuccess) return cuda_fail(e, "decode shared-memory size");
    e = decode_occupancy(p->kind, threads, p->smem, &occ);
  }
  if (e != cudaSuccess) return cuda_fail(e, "decode occupancy");
  if (occ < 1) {
    set_error("decode kernel does not fit an SM (%zu bytes shared memory)", p->smem);
    return FPTC_ERR_UNSUPPORTED;
  }
  p->ctas_per_sm = p->opts.ctas_per_sm ? std::min<uint32_t>(p->opts.ctas_per_sm, (uint32_t)occ) : (uint32_t)occ;
  const uint64_t full = (uint64_t)p->sm_count * p->ctas_per_sm;
  p->grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(full, p->n_tiles));
  // backward (the warp-tile adjoint serves N = 32, E = 16 plans); decided afresh on every
  // configuration: the autotuner configures one candidate after another
  p->b_warp = false;
  if ((p->kind == FPTC_KERNEL_WARP_TILE && !shape) || (p->kind == FPTC_KERNEL_TENSOR && !p->tcs_N)) {
    // the warp-tile adjoint: 16 warps if their buffers fit, else 8
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    p->b_warp = false;
    for (uint32_t t : {512u, 256u}) {
      const size_t need = backward_warp_smem_layout(t, lm.data(), (uint32_t)lm.size(), &p->b_wp);
      if (need <= (size_t)optin) {
        e = backward_warp_smem_config(t, need);
        if (e != cudaSuccess) return cuda_fail(e, "backward shared-memory size");
        p->b_warp = true;
        p->b_threads = t;
        p->b_smem = need;
        p->b_grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)p->sm_count, p->n_tiles));
        return FPTC_OK;
      }
    }
  }
  p->b_threads = (threads == 128 || threads == 256 || threads == 512) ? threads : 256u;  // backward variants
  p->b_smem = backward_smem_bytes(p->b_threads, p->lut_cap, p->coef_cap, p->gx_cap, p->basis_cap);
  e = backward_smem_config(p->b_threads, p->b_smem);
  if (e != cudaSuccess) return cuda_fail(e, "backward shared-memory size");
  int bocc = 0;
  e = backward_occupancy(p->b_threads, p->b_smem, &bocc);
  if (e != cudaSuccess) return cuda_fail(e, "backward occupancy");
  if (bocc < 1) {
    set_error("backward kernel does not fit an SM (%zu bytes shared memory)", p->b_smem);
    return FPTC_ERR_UNSUPPORTED;
  }
  p->b_grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)p->sm_count * bocc, p->n_tiles));
  return FPTC_OK;
}

fptc_status upload_layout(fptc_plan *p) {
  cudaError_t e;
  if (p->d_segs) {
    e = cudaMemcpy(p->d_segs, p->segs.data(), p->segs.size() * sizeof(SegDev), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload segments");
    e = cudaMemcpy(p->d_domains, p->dom_dev.data(), p->dom_dev.size() * sizeof(DomainDev), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload domains");
  }
  if (p->n_tiles > p->tiles_capacity) {
    if (p->d_tiles) {
      cudaFree(p->d_tiles);
      p->device_bytes -= p->tiles_capacity * sizeof(TileRec);
      p->d_tiles = nullptr;
    }
    const uint64_t cap = std::max<uint64_t>(p->n_tiles, 1);
    e = cudaMalloc(&p->d_tiles, cap * sizeof(TileRec));
    if (e != cudaSuccess) return cuda_fail(e, "tile table");
    p->tiles_capacity = cap;
    p->device_bytes += cap * sizeof(TileRec);
  }
  return FPTC_OK;
}

// records: a TileRec per tile for kernels that read one (the warp-tile kernels
// locate their tiles from the chunk offsets and need none).
IndexParams index_params(const fptc_plan *p, const uint8_t *d_symlen, bool records) {
  IndexParams ip{};
  ip.records = records ? 1u : 0u;
  ip.symlen = d_symlen;
  ip.segs = p->d_segs;
  ip.domains = p->d_domains;
  ip.grid = (uint32_t)p->sm_count * 8u;
  ip.chunk_sum = p->d_chunk_sum;
  ip.chunk_off = p->d_chunk_off;
  ip.seg_bad = p->d_seg_bad;
  ip.tiles = p->d_tiles;
  ip.status = p->d_status;
  ip.chunk_begin = 0;
  ip.chunk_end = p->n_chunks;
  ip.seg_begin = 0;
  ip.seg_end = (uint32_t)p->segs.size();
  return ip;
}

// Whether the plan's forward decode reads a record per tile.
bool needs_records(const fptc_plan *p) {
  return !(p->kind == FPTC_KERNEL_WARP_TILE || p->kind == FPTC_KERNEL_TENSOR) ||
         p->opts.schedule == FPTC_SCHEDULE_THREE_KERNEL;
}

DecodeParams decode_params(const fptc_plan *p, const uint64_t *d_words, const uint8_t *d_symlen, float *d_out,
                           uint8_t *d_levels, const float *d_scale) {
  DecodeParams dp{};
  dp.words = d_words;
  dp.symlen = d_symlen;
  dp.out = d_out;
  dp.levels = d_levels;
  dp.scale = d_scale;
  dp.segs = p->d_segs;
  dp.domains = p->d_domains;
  dp.luts = p->d_luts;
  dp.basis = p->d_basis;
  dp.tiles = p->d_tiles;
  dp.chunk_off = p->d_chunk_off;
  dp.seg_bad = p->d_seg_bad;
  dp.status = p->d_status;
  dp.tile_begin = 0;
  dp.tile_end = p->n_tiles;
  dp.seg_begin = 0;
  dp.seg_end = (uint32_t)p->segs.size();
  dp.lut_cap = p->lut_cap;
  dp.coef_cap = p->coef_cap;
  return dp;
}

// Index + decode of queue segments [s0, s1) (tiles and chunks of those segments).
cudaError_t run_range(const fptc_plan *p, const IndexParams &ip0, const DecodeParams &dp0, uint32_t s0, uint32_t s1,
                      bool index, cudaStream_t st, bool decode = true, uint32_t halves = 3u) {
  if (s1 <= s0) return cudaSuccess;
  const SegDev &a = p->segs[s0];
  const SegDev &b = p->segs[s1 - 1];
  if (index) {
    IndexParams ip = ip0;
    ip.seg_begin = s0;
    ip.seg_end = s1;
    ip.chunk_begin = a.chunk_base;
    ip.chunk_end = b.chunk_base + b.n_chunks;
    cudaError_t e = launch_index(ip, st);
    if (e == cudaSuccess && p->opts.schedule == FPTC_SCHEDULE_THREE_KERNEL) e = launch_word_offsets(ip, p->d_word_off, st);
    if (e != cudaSuccess) return e;
  }
  if (!decode) return cudaSuccess;
  DecodeParams dp = dp0;
  dp.seg_begin = s0;
  dp.seg_end = s1;
  dp.tile_begin = a.tile_base;
  dp.tile_end = b.tile_base + b.n_tiles;
  if (p->opts.schedule == FPTC_SCHEDULE_THREE_KERNEL)
    return launch_three_kernel(dp, p->d_word_off, dp.levels ? dp.levels : p->d_lev_scratch, a.chunk_base,
                               b.chunk_base + b.n_chunks, halves, st);
  const uint64_t tiles = dp.tile_end - dp.tile_begin;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(p->grid, tiles));
  if (p->kind == FPTC_KERNEL_BLOCK_TILE) return launch_fixed(dp, p->threads, grid, p->smem, st);
  if (p->kind == FPTC_KERNEL_WARP_TILE) {
    WarpParams wp = p->wp;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    wp.out_tma = encode_out_map(&map, dp.out, p->out_extent) ? 1u : 0u;
    if (p->shape) return launch_shape(dp, wp, map, p->threads, p->shape_any, grid, p->smem, st);
    return launch_warp(dp, wp, map, p->threads, grid, p->smem, st);
  }
  if (p->kind == FPTC_KERNEL_TENSOR && p->tcs_N) {
    WarpParams wp = p->wp;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    wp.out_tma = encode_out_map3(&map, dp.out, p->out_extent, p->tcs_N) ? 1u : 0u;
    return launch_tcs(dp, wp, p->tp, map, p->opts.idct, p->tcs_N, p->tcs_E, grid, p->smem, st);
  }
  if (p->kind == FPTC_KERNEL_TENSOR) {
    WarpParams wp = p->wp;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    wp.out_tma = encode_out_map(&map, dp.out, p->out_extent) ? 1u : 0u;
    return launch_tc(dp, wp, p->tp, map, p->opts.idct, p->threads, grid, p->smem, st);
  }
  return launch_decode(dp, p->kind, p->threads, grid, p->smem, st);
}

fptc_status check_plan(const fptc_plan *p) {
  if (!p) {
    set_error("plan is NULL");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  return FPTC_OK;
}

fptc_status check_ptr(const void *ptr, size_t align, bool needed, const char *name) {
  if (needed && !ptr) {
    set_error("%s is NULL", name);
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  if (ptr && (reinterpret_cast<uintptr_t>(ptr) % align) != 0) {
    set_error("%s must be %zu-byte aligned", name, align);
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  return FPTC_OK;
}

}  // namespace

extern "C" {

uint32_t fptc_abi_version(void) { return FPTC_ABI_VERSION; }

uint64_t fptc_struct_size(uint32_t which) {
  switch (which) {
    case 0: return sizeof(fptc_domain);
    case 1: return sizeof(fptc_segment);
    case 2: return sizeof(fptc_plan_options);
    case 3: return sizeof(fptc_plan_info);
    default: return 0;
  }
}

const char *fptc_status_string(fptc_status s) {
  switch (s) {
    case FPTC_OK: return "ok";
    case FPTC_ERR_INVALID_ARGUMENT: return "invalid argument";
    case FPTC_ERR_UNSUPPORTED: return "unsupported";
    case FPTC_ERR_OUT_OF_MEMORY: return "out of memory";
    case FPTC_ERR_CUDA: return "CUDA error";
    case FPTC_ERR_CORRUPT_STREAM: return "corrupt stream";
  }
  return "unknown status";
}

fptc_status fptc_plan_create(fptc_plan **out, int device, const fptc_domain *domains, uint32_t n_domains,
                             const fptc_segment *segments, uint64_t n_segments, const fptc_plan_options *opts) {
  return guarded([&]() -> fptc_status {
    clear_error();
    if (!out) {
      set_error("plan output pointer is NULL");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    *out = nullptr;
    if (n_domains == 0 || !domains) {
      set_error("at least one domain is required");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (n_segments > 0 && !segments) {
      set_error("segments is NULL");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (n_segments > 0xFFFFFFF0ull) {
      set_error("too many segments");
      return FPTC_ERR_UNSUPPORTED;
    }
    fptc_plan_options o{};
    o.idct = FPTC_IDCT_FP32;
    o.schedule = FPTC_SCHEDULE_PERSISTENT;
    if (opts) o = *opts;
    if (o.idct > FPTC_IDCT_TF32X3 || o.schedule > FPTC_SCHEDULE_THREE_KERNEL || o.reserved[0] || o.reserved[1] ||
        (o.schedule == FPTC_SCHEDULE_THREE_KERNEL && o.idct != FPTC_IDCT_FP32)) {
      set_error("invalid plan options");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    if (o.kernel > FPTC_KERNEL_TENSOR) {
      set_error("unknown kernel %u", o.kernel);
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    bool all_fixed = true, all_shape = n_domains > 0;
    for (uint32_t d = 0; d < n_domains; ++d) {
      all_fixed = all_fixed && domains[d].N == 32 && domains[d].E == 16;
      all_shape = all_shape && shape_supported(domains[d].N);
    }
    const bool fixed_ok = all_fixed && n_domains <= kWarpMaxDomains;
    // other shapes: N in [4, 128] for every domain
    const bool shape_ok = !all_fixed && all_shape && n_domains <= kWarpMaxDomains;
    const bool warp_ok = fixed_ok || shape_ok;
    if ((o.kernel == FPTC_KERNEL_BLOCK_TILE && !all_fixed) || (o.kernel == FPTC_KERNEL_WARP_TILE && !warp_ok)) {
      set_error("the block-tile kernel needs N = 32, E = 16 in every domain; the warp-tile kernel that, or "
                "N in [4, 128] in every domain (at most %u domains)", kWarpMaxDomains);
      return FPTC_ERR_UNSUPPORTED;
    }
    // the tensor-core transform: N = 32, E = 16 in every domain (decode_tc.cu), or one
    // shape with E >= 32 shared by every domain (decode_tcs.cu)
    bool tcs_ok = !all_fixed && n_domains > 0 && n_domains <= kWarpMaxDomains &&
                  tcs_supported(domains[0].N, domains[0].E);
    for (uint32_t d = 1; d < n_domains && tcs_ok; ++d)
      tcs_ok = domains[d].N == domains[0].N && domains[d].E == domains[0].E;
    if (o.idct != FPTC_IDCT_FP32 || o.kernel == FPTC_KERNEL_TENSOR) {
      if (!(fixed_ok || tcs_ok) || o.idct == FPTC_IDCT_FP32) {
        set_error("the tensor-core transform needs N = 32, E = 16 in every domain, or one shape (N, E) in "
                  "{(32, 32), (64, 32), (128, 32), (128, 64)} shared by every domain (at most %u domains), and "
                  "idct = TF32, BF16X3 or TF32X3", kWarpMaxDomains);
        return FPTC_ERR_UNSUPPORTED;
      }
      o.kernel = FPTC_KERNEL_TENSOR;
    }
    if (o.kernel != FPTC_KERNEL_TENSOR) tcs_ok = false;
    if (o.kernel == FPTC_KERNEL_AUTO) {
      // the warp-tile kernel keeps every domain's tables in shared memory: it is
      // the default when they fit beside at least four warps' buffers
      bool fits = false;
      if (warp_ok) {
        std::vector<uint32_t> lm(n_domains);
        for (uint32_t d = 0; d < n_domains; ++d) lm[d] = domains[d].lmax;
        WarpParams probe{};
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) optin = 0;
        if (fixed_ok) {
          fits = warp_smem_layout(128, lm.data(), n_domains, &probe) <= (size_t)optin;
        } else {
          std::vector<uint32_t> ns(n_domains), es(n_domains);
          for (uint32_t d = 0; d < n_domains; ++d) {
            ns[d] = domains[d].N;
            es[d] = domains[d].E;
          }
          fits = shape_smem_layout(256, lm.data(), ns.data(), es.data(), n_domains, &probe) <= (size_t)optin;
        }
      }
      o.kernel = fits ? FPTC_KERNEL_WARP_TILE : (all_fixed ? FPTC_KERNEL_BLOCK_TILE : FPTC_KERNEL_GENERIC);
    }
    if (o.kernel == FPTC_KERNEL_WARP_TILE) o.tile_samples = shape_ok ? 0 : warp_tile_windows() * 32;
    if (o.kernel == FPTC_KERNEL_TENSOR)
      o.tile_samples = tcs_ok ? tcs_tile_windows(domains[0].E) * domains[0].N : tc_tile_windows() * 32;
    if (o.tile_samples == 0) o.tile_samples = o.kernel == FPTC_KERNEL_BLOCK_TILE ? 8192 : 4096;
    if (o.tile_samples > 65536) {
      set_error("tile_samples must be <= 65536");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    for (uint32_t d = 0; d < n_domains; ++d) {
      fptc_status st = fptc_validate_domain(&domains[d]);
      if (st != FPTC_OK) {
        std::string m = fptc_last_error_message();
        set_error("domain %u: %s", d, m.c_str());
        return st;
      }
    }

    // the plan under construction: released into *out only on success, so that
    // an error return or an exception frees what it holds
    std::unique_ptr<fptc_plan, PlanDeleter> owner(new (std::nothrow) fptc_plan());
    if (!owner) return FPTC_ERR_OUT_OF_MEMORY;
    fptc_plan *const p = owner.get();
    p->device = device;
    p->opts = o;
    p->domains.assign(domains, domains + n_domains);
    p->caller_segs.assign(segments, segments + n_segments);

    // ---- segment metadata checks
    std::vector<std::pair<uint64_t, uint64_t>> out_ranges;
    for (uint64_t i = 0; i < n_segments; ++i) {
      const fptc_segment &s = segments[i];
      if (s.domain >= n_domains || s.reserved != 0) {
        set_error("segment %llu: domain %u out of range", (unsigned long long)i, s.domain);
        return FPTC_ERR_INVALID_ARGUMENT;
      }
      const fptc_domain &d = domains[s.domain];
      const uint64_t W = (s.n_samples + d.N - 1) / d.N;
      const uint64_t L = W * d.E;
      // each word holds 1..64 codewords (Alg. 1 never closes an empty word)
      const uint64_t min_words = (L + 63) / 64;
      if (s.n_words < min_words || s.n_words > L) {
        set_error("segment %llu: %llu words cannot hold %llu symbols", (unsigned long long)i,
                  (unsigned long long)s.n_words, (unsigned long long)L);
        return FPTC_ERR_INVALID_ARGUMENT;
      }
      if (s.word_offset + s.n_words < s.word_offset || s.out_offset + s.n_samples < s.out_offset) {
        set_error("segment %llu: offset overflow", (unsigned long long)i);
        return FPTC_ERR_INVALID_ARGUMENT;
      }
      p->words_extent = std::max(p->words_extent, s.word_offset + s.n_words);
      p->out_extent = std::max(p->out_extent, s.out_offset + s.n_samples);
      p->n_samples += s.n_samples;
      p->n_words += s.n_words;
      if (s.n_samples) out_ranges.push_back({s.out_offset, s.out_offset + s.n_samples});
    }
    std::sort(out_ranges.begin(), out_ranges.end());
    for (size_t i = 1; i < out_ranges.size(); ++i) {
      if (out_ranges[i].first < out_ranges[i - 1].second) {
        set_error("segment output ranges overlap");
        return FPTC_ERR_INVALID_ARGUMENT;
      }
    }

    // ---- per-domain tables on the host
    p->dom_dev.resize(n_domains);
    std::vector<uint16_t> luts;
    std::vector<float> basis;
    uint32_t max_lmax = 1;
    p->basis_cap = 0;
    for (uint32_t d = 0; d < n_domains; ++d) {
      const fptc_domain &dm = domains[d];
      DomainDev &dd = p->dom_dev[d];
      fill_domain_dev(dm, &dd);
      max_lmax = std::max(max_lmax, dm.lmax);
      while (luts.size() % 8) luts.push_back(0);  // 16-byte aligned table starts
      dd.lut_offset = (uint32_t)luts.size();
      luts.resize(luts.size() + (size_t(1) << dm.lmax));
      fptc_build_decode_table(&dm, luts.data() + dd.lut_offset);
      while (basis.size() % 4) basis.push_back(0.f);
      dd.basis_offset = (uint32_t)basis.size();
      for (uint32_t k = 0; k < dm.E; ++k)
        for (uint32_t n = 0; n < dm.N; ++n) basis.push_back(basis_value(dm.N, n, k));
      p->basis_cap = std::max(p->basis_cap, dm.N * dm.E);
    }
    p->lut_cap = 1u << max_lmax;
    p->kind = (int)o.kernel;
    p->shape = shape_ok;
    p->shape_any = false;
    for (uint32_t d = 0; d < n_domains; ++d) p->shape_any = p->shape_any || !shape_pow2_only(domains[d].N);
    p->tcs_N = tcs_ok ? domains[0].N : 0u;
    p->tcs_E = tcs_ok ? domains[0].E : 0u;

    // ---- tile queue: segments ordered by output offset
    p->queue.resize(n_segments);
    std::iota(p->queue.begin(), p->queue.end(), 0u);
    std::stable_sort(p->queue.begin(), p->queue.end(), [&](uint32_t a, uint32_t b) {
      return segments[a].out_offset < segments[b].out_offset;
    });
    p->level_off.resize(n_segments);
    uint64_t lv = 0;
    for (uint64_t i = 0; i < n_segments; ++i) {
      const fptc_domain &d = domains[segments[i].domain];
      p->level_off[i] = lv;
      lv += (segments[i].n_samples + d.N - 1) / d.N * d.E;
    }
    p->n_levels = lv;
    p->segs.resize(n_segments);
    uint64_t chunk = 0;
    for (uint64_t qi = 0; qi < n_segments; ++qi) {
      const uint32_t ci = p->queue[qi];
      const fptc_segment &s = segments[ci];
      const fptc_domain &d = domains[s.domain];
      SegDev &sd = p->segs[qi];
      std::memset(&sd, 0, sizeof(sd));
      sd.word_offset = s.word_offset;
      sd.n_words = s.n_words;
      sd.n_samples = s.n_samples;
      sd.out_offset = s.out_offset;
      sd.level_offset = p->level_off[ci];
      sd.n_windows = (s.n_samples + d.N - 1) / d.N;
      sd.domain = s.domain;
      sd.caller_index = ci;
      sd.out_aligned = ((s.out_offset % 4) == 0 ? 1u : 0u) | ((s.out_offset % 8) == 0 ? 2u : 0u) |
                       ((s.out_offset % 32) == 0 ? 4u : 0u);
      sd.chunk_base = chunk;
      sd.n_chunks = (uint32_t)chunks_of(s.n_words);
      chunk += sd.n_chunks;
    }
    p->n_chunks = chunk;
    layout_tiles(p, o.tile_samples);

    // ---- device
    fptc_status st = FPTC_OK;
    {
      DeviceGuard g(device);
      if (!g.ok) {
        set_error("cannot select device %d", device);
        return FPTC_ERR_CUDA;
      }
      cudaError_t e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, device);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "device query");
        return st;
      }
      size_t b = 0;
      if ((e = upload(&p->d_domains, p->dom_dev, &b)) != cudaSuccess ||
          (e = upload(&p->d_segs, p->segs, &b)) != cudaSuccess ||
          (e = upload(&p->d_luts, luts, &b)) != cudaSuccess || (e = upload(&p->d_basis, basis, &b)) != cudaSuccess) {
        st = cuda_fail(e, "plan upload");
      }
      if (st == FPTC_OK) {
        const size_t nc = std::max<uint64_t>(p->n_chunks, 1), ns = std::max<uint64_t>(n_segments, 1);
        if ((e = cudaMalloc(&p->d_chunk_sum, nc * 4)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_chunk_off, nc * 8)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_seg_bad, ns * 4)) != cudaSuccess ||
            (e = cudaMalloc(&p->d_status, sizeof(DevStatus))) != cudaSuccess) {
          st = cuda_fail(e, "plan scratch");
        } else {
          b += nc * 12 + ns * 4 + sizeof(DevStatus);
          DevStatus s0{0u, 0u, ~0ull};
          e = cudaMemcpy(p->d_status, &s0, sizeof(s0), cudaMemcpyHostToDevice);
          if (e == cudaSuccess) e = cudaMemset(p->d_seg_bad, 0, ns * 4);
          if (e == cudaSuccess && o.schedule == FPTC_SCHEDULE_THREE_KERNEL) {
            e = cudaMalloc(&p->d_word_off, std::max<uint64_t>(p->words_extent, 1) * 4);
            if (e == cudaSuccess) e = cudaMalloc(&p->d_lev_scratch, std::max<uint64_t>(p->n_levels, 1));
            if (e == cudaSuccess) b += std::max<uint64_t>(p->words_extent, 1) * 4 + std::max<uint64_t>(p->n_levels, 1);
          }
          if (e != cudaSuccess) st = cuda_fail(e, "plan scratch init");
        }
      }
      p->device_bytes = b;
      if (st == FPTC_OK) st = upload_layout(p);
      if (st == FPTC_OK) st = configure_launch(p);
      if (st == FPTC_OK) {
        for (auto &a : p->aux)
          if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->up, cudaStreamNonBlocking);
        for (auto &v : p->ev)
          if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
        for (auto &v : p->evh)
          if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
        if (e != cudaSuccess)
          st = cuda_fail(e, "plan streams");
      }
      if (st != FPTC_OK) return st;
    }
    *out = owner.release();
    return FPTC_OK;
  });
}

void fptc_plan_destroy(fptc_plan *p) {
  if (!p) return;
  {
    DeviceGuard g(p->device);
    cudaDeviceSynchronize();
  }
  PlanDeleter()(p);
}

fptc_status fptc_plan_get_info(const fptc_plan *p, fptc_plan_info *info) {
  if (check_plan(p) != FPTC_OK || !info) return FPTC_ERR_INVALID_ARGUMENT;
  std::memset(info, 0, sizeof(*info));
  info->n_segments = p->segs.size();
  info->n_tiles = p->n_tiles;
  info->n_chunks = p->n_chunks;
  info->words_extent = p->words_extent;
  info->out_extent = p->out_extent;
  info->n_samples_total = p->n_samples;
  info->n_words_total = p->n_words;
  info->n_levels_total = p->n_levels;
  info->device_bytes = p->device_bytes;
  info->n_domains = (uint32_t)p->domains.size();
  info->device = (uint32_t)p->device;
  info->sm_count = (uint32_t)p->sm_count;
  info->threads = p->threads;
  info->grid = p->grid;
  info->ctas_per_sm = p->ctas_per_sm;
  info->idct = p->opts.idct;
  info->schedule = p->opts.schedule;
  info->kernel = (uint32_t)p->kind;
  info->smem_bytes = (uint32_t)p->smem;
  return FPTC_OK;
}

fptc_status fptc_plan_level_offsets(const fptc_plan *p, uint64_t *offsets) {
  return guarded([&]() -> fptc_status {
    if (check_plan(p) != FPTC_OK) return FPTC_ERR_INVALID_ARGUMENT;
    if (!offsets && !p->level_off.empty()) {
      set_error("offsets is NULL");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    std::copy(p->level_off.begin(), p->level_off.end(), offsets);
    return FPTC_OK;
  });
}

uint32_t fptc_plan_launches_per_decode(const fptc_plan *p) {
  if (!p) return 0;
  if (p->segs.empty()) return 0;
  if (p->opts.schedule == FPTC_SCHEDULE_PERSISTENT) return (p->n_chunks ? 3u : 1u) + 1u;
  if (p->opts.schedule == FPTC_SCHEDULE_THREE_KERNEL) return (p->n_chunks ? 4u : 1u) + (p->n_chunks ? 2u : 1u);
  uint32_t n = 0;
  for (const auto &s : p->segs) n += (s.n_chunks ? 3u : 1u) + 1u;
  return n;
}

fptc_status fptc_decode_stages(fptc_plan *p, const uint64_t *d_words, const uint8_t *d_symlen, float *d_out,
                               uint8_t *d_levels, const float *d_scale, uint32_t stages, fptc_stream stream) {
  clear_error();
  fptc_status st = check_plan(p);
  if (st != FPTC_OK) return st;
  if (stages & ~(FPTC_STAGE_INDEX | FPTC_STAGE_DECODE | FPTC_STAGE_LOSSLESS | FPTC_STAGE_LOSSY)) {
    set_error("unknown stage bits 0x%x", stages);
    return FPTC_ERR_INVALID_ARGUMENT;
  }
  if ((stages & (FPTC_STAGE_LOSSLESS | FPTC_STAGE_LOSSY)) && p->opts.schedule != FPTC_SCHEDULE_THREE_KERNEL) {
    set_error("the lossless and lossy stages run on their own only in the three-kernel schedule");
    return FPTC_ERR_UNSUPPORTED;
  }
  if (p->segs.empty() || !stages) return FPTC_OK;
  // decode halves of the three-kernel schedule: bit 0 lossless, bit 1 lossy
  const uint32_t halves = (stages & FPTC_STAGE_DECODE ? 3u : 0u) | (stages & FPTC_STAGE_LOSSLESS ? 1u : 0u) |
                          (stages & FPTC_STAGE_LOSSY ? 2u : 0u);
  const bool idx = stages & FPTC_STAGE_INDEX, dec = halves != 0;
  if ((st = check_ptr(d_words, 8, dec && p->words_extent > 0, "d_words")) != FPTC_OK ||
      (st = check_ptr(d_symlen, 1, p->words_extent > 0, "d_symlen")) != FPTC_OK ||
      (st = check_ptr(d_out, 16, dec && p->out_extent > 0, "d_out")) != FPTC_OK ||
      (st = check_ptr(d_scale, 4, false, "d_scale")) != FPTC_OK)
    return st;
  DeviceGuard g(p->device);
  if (!g.ok) return cuda_fail(cudaGetLastError(), "set device");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const IndexParams ip = index_params(p, d_symlen, needs_records(p));
  const DecodeParams dp = decode_params(p, d_words, d_symlen, d_out, d_levels, d_scale);
  cudaError_t e = cudaSuccess;
  if (p->opts.schedule != FPTC_SCHEDULE_PER_SEGMENT) {
    e = run_range(p, ip, dp, 0, (uint32_t)p->segs.size(), idx, s, dec, halves);
  } else {
    for (uint32_t i = 0; i < p->segs.size() && e == cudaSuccess; ++i) e = run_range(p, ip, dp, i, i + 1, idx, s, dec);
  }
  if (e != cudaSuccess) return cuda_fail(e, "decode launch");
  return FPTC_OK;
}

fptc_status fptc_decode_batch(fptc_plan *p, const uint64_t *d_words, const uint8_t *d_symlen, float *d_out,
                              uint8_t *d_levels, const float *d_scale, fptc_stream stream) {
  return fptc_decode_stages(p, d_words, d_symlen, d_out, d_levels, d_scale, FPTC_STAGE_INDEX | FPTC_STAGE_DECODE,
                            stream);
}

fptc_status fptc_decode_backward(fptc_plan *p, const uint64_t *d_words, const uint8_t *d_symlen,
                                 const uint8_t *d_levels, const float *d_scale, const float *d_grad_out,
                                 float *d_grad_coeffs, double *d_grad_scale, fptc_stream stream) {
  clear_error();
  fptc_status st = check_plan(p);
  if (st != FPTC_OK) return st;
  const bool redecode = d_levels == nullptr;
  if ((st = check_ptr(d_grad_scale, 8, true, "d_grad_scale")) != FPTC_OK ||
      (st = check_ptr(d_words, 8, redecode && p->words_extent > 0, "d_words")) != FPTC_OK ||
      (st = check_ptr(d_symlen, 1, redecode && p->words_extent > 0, "d_symlen")) != FPTC_OK ||
      (st = check_ptr(d_grad_out, 4, p->out_extent > 0, "d_grad_out")) != FPTC_OK ||
      (st = check_ptr(d_grad_coeffs, 4, false, "d_grad_coeffs")) != FPTC_OK ||
      (st = check_ptr(d_scale, 4, false, "d_scale")) != FPTC_OK)
    return st;
  DeviceGuard g(p->device);
  if (!g.ok) return cuda_fail(cudaGetLastError(), "set device");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(d_grad_scale, 0, p->domains.size() * 3 * sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e, "zero grad_scale");
  if (p->segs.empty()) return FPTC_OK;
  if (redecode) {
    e = launch_index(index_params(p, d_symlen, !p->b_warp), s);
    if (e != cudaSuccess) return cuda_fail(e, "index launch");
  }
  BackwardParams bp{};
  bp.d = decode_params(p, d_words, d_symlen, nullptr, nullptr, d_scale);
  bp.levels_in = d_levels;
  bp.grad_out = d_grad_out;
  bp.grad_coeffs = d_grad_coeffs;
  bp.grad_scale = d_grad_scale;
  bp.gx_cap = p->gx_cap;
  bp.basis_cap = p->basis_cap;
  if (p->b_warp) {
    WarpParams wp = p->b_wp;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    wp.out_tma = encode_out_map(&map, const_cast<float *>(d_grad_out), p->out_extent) ? 1u : 0u;
    e = launch_backward_warp(bp, wp, map, p->b_threads, p->b_grid, p->b_smem, s);
  } else {
    e = launch_backward(bp, p->b_threads, p->b_grid, p->b_smem, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return FPTC_OK;
}

fptc_status fptc_decode_host(fptc_plan *p, const uint64_t *h_words, const uint8_t *h_symlen, float *h_out,
                             uint64_t *d_words, uint8_t *d_symlen, float *d_out, fptc_stream stream) {
  return guarded([&]() -> fptc_status {
    clear_error();
    fptc_status st = check_plan(p);
    if (st != FPTC_OK) return st;
    if (p->segs.empty()) return FPTC_OK;
    const bool any_words = p->words_extent > 0, any_out = p->out_extent > 0;
    if ((st = check_ptr(h_words, 8, any_words, "h_words")) != FPTC_OK ||
        (st = check_ptr(h_symlen, 1, any_words, "h_symlen")) != FPTC_OK ||
        (st = check_ptr(h_out, 4, any_out, "h_out")) != FPTC_OK ||
        (st = check_ptr(d_words, 8, any_words, "d_words")) != FPTC_OK ||
        (st = check_ptr(d_symlen, 1, any_words, "d_symlen")) != FPTC_OK ||
        (st = check_ptr(d_out, 16, any_out, "d_out")) != FPTC_OK)
      return st;
    DeviceGuard g(p->device);
    if (!g.ok) return cuda_fail(cudaGetLastError(), "set device");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Pieces of about equal output in queue (output) order.  Piece k's words go
    // up on the upload stream, it is indexed and decoded on `stream` once they
    // are there, and its samples go back on one of the copy-back streams, so
    // uploads, decoding and copies back of different pieces overlap.
    struct Piece {
      uint32_t s0, s1;
      uint64_t w0, w1;  // hull of the piece's words
      uint64_t o0, o1;  // hull of its output
    };
    std::vector<Piece> pieces;
    {
      const uint32_t n = (uint32_t)p->segs.size();
      const uint64_t per = (p->n_samples + fptc_plan::kPieces - 1) / fptc_plan::kPieces;
      uint32_t s0 = 0;
      while (s0 < n) {
        uint32_t s1 = s0;
        uint64_t acc = 0;
        while (s1 < n && (acc < per || s1 == s0)) acc += p->segs[s1++].n_samples;
        if (pieces.size() == fptc_plan::kPieces - 1) s1 = n;  // the last piece takes the rest
        Piece pc{s0, s1, UINT64_MAX, 0, UINT64_MAX, 0};
        for (uint32_t i = s0; i < s1; ++i) {
          const SegDev &sg = p->segs[i];
          if (sg.n_words) {
            pc.w0 = std::min(pc.w0, sg.word_offset);
            pc.w1 = std::max(pc.w1, sg.word_offset + sg.n_words);
          }
          if (sg.n_samples) {
            pc.o0 = std::min(pc.o0, sg.out_offset);
            pc.o1 = std::max(pc.o1, sg.out_offset + sg.n_samples);
          }
        }
        pieces.push_back(pc);
        s0 = s1;
      }
    }
    // uploads per piece only where the pieces' word hulls are disjoint and ascending
    // (words laid out in output order); otherwise every word goes up first
    bool split_up = true;
    {
      uint64_t end = 0;
      for (const Piece &pc : pieces)
        if (pc.w1 > pc.w0) {
          split_up = split_up && pc.w0 >= end;
          end = pc.w1;
        }
    }
    auto upload = [&](uint64_t w0, uint64_t w1) -> cudaError_t {
      if (w1 <= w0) return cudaSuccess;
      cudaError_t r = cudaMemcpyAsync(d_words + w0, h_words + w0, (w1 - w0) * 8, cudaMemcpyHostToDevice, p->up);
      if (r == cudaSuccess) r = cudaMemcpyAsync(d_symlen + w0, h_symlen + w0, w1 - w0, cudaMemcpyHostToDevice, p->up);
      return r;
    };
    // the device buffers are the caller's: uploads start after the work already on `stream`
    cudaError_t e = cudaEventRecord(p->ev_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->up, p->ev_start, 0);
    if (e == cudaSuccess && any_words && !split_up) e = upload(0, p->words_extent);
    if (e != cudaSuccess) return cuda_fail(e, "copy to device");
    const IndexParams ip = index_params(p, d_symlen, needs_records(p));
    const DecodeParams dp = decode_params(p, d_words, d_symlen, d_out, nullptr, nullptr);
    for (size_t k = 0; k < pieces.size() && e == cudaSuccess; ++k) {
      const Piece &pc = pieces[k];
      if (split_up) e = upload(pc.w0, pc.w1);
      if (e == cudaSuccess) e = cudaEventRecord(p->evh[k], p->up);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->evh[k], 0);
      if (e == cudaSuccess) e = run_range(p, ip, dp, pc.s0, pc.s1, true, s);
      if (e != cudaSuccess) break;
      cudaStream_t a = p->aux[k % fptc_plan::kAux];
      if ((e = cudaEventRecord(p->ev[k], s)) != cudaSuccess) break;
      if ((e = cudaStreamWaitEvent(a, p->ev[k], 0)) != cudaSuccess) break;
      if (pc.o1 > pc.o0)
        e = cudaMemcpyAsync(h_out + pc.o0, d_out + pc.o0, (pc.o1 - pc.o0) * 4, cudaMemcpyDeviceToHost, a);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->up);
    for (auto &a : p->aux)
      if (e == cudaSuccess) e = cudaStreamSynchronize(a);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "end-to-end decode");
    return FPTC_OK;
  });
}

fptc_status fptc_plan_device_status(fptc_plan *p, uint32_t *flags, uint64_t *first_bad) {
  clear_error();
  fptc_status st = check_plan(p);
  if (st != FPTC_OK) return st;
  DeviceGuard g(p->device);
  cudaError_t e = cudaDeviceSynchronize();
  DevStatus h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, p->d_status, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    DevStatus s0{0u, 0u, ~0ull};
    e = cudaMemcpy(p->d_status, &s0, sizeof(s0), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_fail(e, "read device status");
  if (flags) *flags = h.flags;
  if (first_bad) *first_bad = h.flags ? (uint64_t)h.first_bad : UINT64_MAX;
  if (h.flags) {
    set_error("device found a malformed stream (flags 0x%x, first segment %llu)", h.flags,
              (unsigned long long)h.first_bad);
    return FPTC_ERR_CORRUPT_STREAM;
  }
  return FPTC_OK;
}

fptc_status fptc_plan_autotune(fptc_plan *p, const uint64_t *d_words, const uint8_t *d_symlen, float *d_out,
                               uint32_t trials, fptc_stream stream, fptc_plan_options *best, float *best_ms) {
  return guarded([&]() -> fptc_status {
    clear_error();
    fptc_status st = check_plan(p);
    if (st != FPTC_OK) return st;
    if (trials == 0) trials = 3;
    DeviceGuard g(p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const fptc_plan_options keep = p->opts;
    const int keep_kind = p->kind;
    bool fixed = true;
    for (const auto &d : p->domains) fixed = fixed && d.N == 32 && d.E == 16;
    struct Cand {
      uint32_t kernel, tile_samples, threads;
    };
    std::vector<Cand> cands;
    if (keep.idct != FPTC_IDCT_FP32 && p->tcs_N)  // the shape kernel: one configuration
      cands.push_back({FPTC_KERNEL_TENSOR, tcs_tile_windows(p->tcs_E) * p->tcs_N, 0u});
    else if (keep.idct != FPTC_IDCT_FP32)
      for (uint32_t th : {256u, 384u, 512u, 640u, 768u, 896u})
        cands.push_back({FPTC_KERNEL_TENSOR, tc_tile_windows() * 32, th});
    for (uint32_t th : {128u, 256u, 512u, 768u, 896u, 1024u}) {
      if (keep.idct != FPTC_IDCT_FP32) continue;
      if (th > 512) {
        if (fixed && p->domains.size() <= kWarpMaxDomains)
          cands.push_back({FPTC_KERNEL_WARP_TILE, warp_tile_windows() * 32, th});
        if (p->shape && th == 768) cands.push_back({FPTC_KERNEL_WARP_TILE, 4096, th});
        continue;
      }
      if (fixed && p->domains.size() <= kWarpMaxDomains)
        cands.push_back({FPTC_KERNEL_WARP_TILE, warp_tile_windows() * 32, th});
      if (p->shape && th >= 256) cands.push_back({FPTC_KERNEL_WARP_TILE, 4096, th});
      if (fixed)
        for (uint32_t ts : {4096u, 8192u}) cands.push_back({FPTC_KERNEL_BLOCK_TILE, ts, th});
      else
        for (uint32_t ts : {2048u, 4096u, 8192u}) cands.push_back({FPTC_KERNEL_GENERIC, ts, th});
    }
    fptc_plan_options win = keep;
    int win_kind = keep_kind;
    float win_ms = 1e30f;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (const Cand &c : cands) {
      p->opts = keep;
      p->opts.kernel = c.kernel;
      p->opts.tile_samples = c.tile_samples;
      p->opts.threads = c.threads;
      p->opts.ctas_per_sm = 0;
      p->kind = (int)c.kernel;
      layout_tiles(p, c.tile_samples);
      if (upload_layout(p) != FPTC_OK || configure_launch(p) != FPTC_OK) continue;
      if (fptc_decode_batch(p, d_words, d_symlen, d_out, nullptr, nullptr, stream) != FPTC_OK) continue;
      std::vector<float> ms;
      for (uint32_t t = 0; t < trials; ++t) {
        cudaEventRecord(a, s);
        fptc_decode_batch(p, d_words, d_symlen, d_out, nullptr, nullptr, stream);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float m = 0;
        cudaEventElapsedTime(&m, a, b);
        ms.push_back(m);
      }
      std::sort(ms.begin(), ms.end());
      const float med = ms[ms.size() / 2];
      if (med < win_ms) {
        win_ms = med;
        win = p->opts;
        win_kind = p->kind;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    p->opts = win;
    p->kind = win_kind;
    layout_tiles(p, win.tile_samples);
    st = upload_layout(p);
    if (st == FPTC_OK) st = configure_launch(p);
    if (st != FPTC_OK) return st;
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    return FPTC_OK;
  });
}

}  // extern "C"
