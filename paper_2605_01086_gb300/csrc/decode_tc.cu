// Fused decode with the inverse DCT on the 5th-generation tensor cores
// (tcgen05, accumulator in tensor memory), for the Table 1 shape N = 32, E = 16.
//
// The SymLen decode, the level staging, the dequantization and the output path
// are those of the warp-tile kernel (warp_tile.cuh): each warp decodes whole
// tiles of 128 windows into level bytes, over a contiguous tile range of its
// own.  The inverse transform of Eq. 1 is
//      D[128 windows x 32 samples] = C[128 x 16 bins] * B[16 x 32]
// with B[k][n] = cos(pi/N (n + 1/2) k) (B[0][n] = 1/2), one product per
// transform step of a warpgroup: its four warps each contribute 32 windows
// (one step of their own current tile) as rows 32 q .. 32 q + 31 of the A
// operand, which lane i of warp q writes straight into tensor-memory lane
// 32 q + i (tcgen05.st: no shared-memory operand, so 28 warps fit); one thread
// issues tcgen05.mma (M = 128, N = 32) with A and D in tensor memory and B in
// shared memory, tcgen05.commit signals an mbarrier, and warp q reads rows
// 32 q .. 32 q + 31 of D with tcgen05.ld 32x32b (lane i = one window: the
// layout the TMA output staging expects).  The A rows of step k + 1 are
// written while product k runs (two A buffers); D is read back before the
// next product is issued.
//
// Precision forms (the integer decode is exact in every form):
//   TF32    one product, operands rounded to TF32 (10-bit mantissa);
//   TF32X3  C = C_big + C_small, B = B_big + B_small (TF32 each), three
//           products C_big B_big + C_big B_small + C_small B_big;
//   BF16X3  the same split with BF16 halves, C_hi B_hi + C_lo B_hi + C_hi B_lo.
// All accumulate in FP32.
//
// Operands: A in tensor memory, one row per lane, K packed along 32-bit
// columns (two BF16 or one TF32 per column).  B in shared memory, K-major, no
// swizzle: a core matrix is 8 rows x 16 bytes stored contiguously; LBO = byte
// distance between core matrices adjacent in K, SBO = between core matrices
// adjacent in N.  A kernel that uses tensor memory runs one CTA per SM.  Every wait on an mbarrier is bounded; on
// expiry the kernel flags FPTC_FLAG_TIMEOUT and the warpgroup stops.
#include "tc_ops.cuh"

namespace fptc {
namespace {

using namespace wt;
using namespace tcx;


template <int MODE, int NWG>
__global__ void __launch_bounds__(NWG * 128, 1) k_decode_tc(const DecodeParams p, const WarpParams wp,
                                                            const TcParams tp,
                                                            const __grid_constant__ CUtensorMap out_map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int WARPS = NWG * 4;
  const DomW *const dw = reinterpret_cast<const DomW *>(smem_raw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wg = warp >> 2, wq = warp & 3;

  // ---- tables, B operand(s), barriers, tensor memory
  load_domain_tables<WARPS * 32>(p, wp.n_domains, smem_raw);
  unsigned char *const b_base = smem_raw + tp.b_off;
  // the same basis for every N = 32, E = 16 domain
  fill_b_operand<MODE>(b_base, p.basis + p.domains[0].basis_offset, threadIdx.x, WARPS * 32);
  uint64_t *const mbar = reinterpret_cast<uint64_t *>(smem_raw + tp.misc_off);  // [NWG]
  uint32_t *const tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + tp.misc_off + 8 * NWG);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NWG; ++i) mbar_init(smem_addr(mbar + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // tensor memory: per warpgroup one D and two A sets, rounded up to a power of two
  constexpr uint32_t kNeed = NWG * wg_cols<MODE>();
  constexpr uint32_t kCols = kNeed <= 32 ? 32u : kNeed <= 64 ? 64u : kNeed <= 128 ? 128u : kNeed <= 256 ? 256u : 512u;
  static_assert(kNeed <= 512, "tensor memory holds 512 columns");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_shared();  // B operand written by threads, read by the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t d_tmem = tmem + wg * wg_cols<MODE>();    // this warpgroup's D, then its two A sets
  const uint32_t a_tmem = d_tmem + 32u;
  const uint32_t lane_off = (wq * 32u) << 16;              // lanes 32 wq .. 32 wq + 31

  unsigned char *const wbase = smem_raw + wp.warp_off + warp * kMiscBytes;
  uint64_t *const wbuf = reinterpret_cast<uint64_t *>(wbase);
  uint8_t *const stage = wbase + kStageOff;
  const uintptr_t tiles0 = (reinterpret_cast<uintptr_t>(smem_raw + tp.tiles_off) + 1023) & ~uintptr_t(1023);
  unsigned char *const otile = reinterpret_cast<unsigned char *>(tiles0) + warp * kOutTile;
  const bool want_lev = p.levels != nullptr;
  const bool vec32_base = (reinterpret_cast<uintptr_t>(p.out) & 31u) == 0;

  // ---- this warp's tiles: an even split of the launch's tile range over all
  // warps; the warpgroup runs as many rounds as its longest range (the four
  // differ by at most one tile), a warp past its range contributing zero rows
  const uint64_t units = (uint64_t)gridDim.x * NWG * 4, u0 = ((uint64_t)blockIdx.x * NWG + wg) * 4;
  uint64_t t0, t1;
  unit_tiles(p, u0 + wq, units, t0, t1);
  uint64_t rounds = 0;
  for (uint32_t q = 0; q < 4; ++q) {
    uint64_t a, b;
    unit_tiles(p, u0 + q, units, a, b);
    rounds = b - a > rounds ? b - a : rounds;
  }

  uint32_t s = find_segment(p.segs, p.seg_begin, p.seg_end, t0 < t1 ? t0 : p.tile_begin);
  uint32_t pn = 0;
  Ctx nxt{0, 0, 0, s, 0};
  if (t0 < t1) {  // where tile t0 starts, then its first words
    nxt = first_ctx(p, s, t0, lane);
    pn = fetch_pass0(p, nxt, lane, wbuf);
  }

  uint32_t phase = 0u;
  bool timeout = false;  // this warp saw an expired wait
  bool stop = false;     // some warp of the warpgroup did (decided at a warpgroup barrier: uniform)
  bool tma_pending = false;
  StepOut prev{0, nullptr, 0, 0, 0};
  uint64_t k = 0;  // steps issued by this warpgroup

  // Reads back the product in D (step k - 1) and stores its windows.
  auto drain = [&](const StepOut &o) {
    {
      const bool late = !mbar_wait(smem_addr(mbar + wg), phase);
      phase ^= 1u;
      timeout = timeout || __any_sync(0xffffffffu, late);  // one decision for the warp
    }
    if (timeout) return;
    tc_fence_after();
    if (o.nwin == 0) return;  // nothing of this product is stored (D is not read)
    const bool tma = (o.flags & 4u) && o.nwin == kStepWin && (uint64_t)kStepWin * kN <= o.left;
    if (tma && tma_pending) {
      if (lane == 0) tma_wait_read();
      __syncwarp();
    }
    unsigned char *const row = otile + lane * (kN * 4);
    const uint32_t sx = lane & 7u;
    const uint64_t s0 = (uint64_t)lane * kN;
    float *const dst = o.dst + s0;
    // the 32 samples of this lane's window, read back 16 at a time (fewer live registers)
#pragma unroll
    for (uint32_t h = 0; h < 2; ++h) {
      uint32_t v[16];
      tmem_ld16(d_tmem + lane_off + 16u * h, v);
      if (tma) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4 *>(row + (((4u * h + q) ^ sx) << 4)) =
              make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else if (lane < o.nwin) {
        if (s0 + kN <= o.left && (o.flags & 2u)) {
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const float vv[8] = {__uint_as_float(v[8 * b]),     __uint_as_float(v[8 * b + 1]),
                                 __uint_as_float(v[8 * b + 2]), __uint_as_float(v[8 * b + 3]),
                                 __uint_as_float(v[8 * b + 4]), __uint_as_float(v[8 * b + 5]),
                                 __uint_as_float(v[8 * b + 6]), __uint_as_float(v[8 * b + 7])};
            st_cs_v8(dst + 16 * h + 8 * b, vv);
          }
        } else if (s0 + kN <= o.left && (o.flags & 1u)) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            __stcs(reinterpret_cast<float4 *>(dst + 16 * h) + j,
                   make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                               __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3])));
        } else {
#pragma unroll
          for (int n = 0; n < 16; ++n)
            if (s0 + 16 * h + n < o.left) dst[16 * h + n] = __uint_as_float(v[n]);
        }
      }
    }
    if (tma) {
      fence_async_shared();
      __syncwarp();
      if (lane == 0) tma_store_rows(&out_map, otile, (int32_t)o.out_row);
      tma_pending = true;
    }
  };

  for (uint64_t r = 0; r < rounds && !stop; ++r) {
    const uint64_t g = t0 + r;
    const bool have = g < t1;
    Ctx cur{0, 0, 0, s, 0};
    uint64_t w[kWPL] = {0, 0};
    uint32_t n[kWPL] = {0, 0};
    if (have) {
      cp_async_wait_all();
      __syncwarp();
      cur = nxt;
      s = cur.seg;
#pragma unroll
      for (int u = 0; u < kWPL; ++u) {
        w[u] = wbuf[kWPL * lane + u];
        n[u] = (pn >> (8 * u)) & 0xffu;
      }
      __syncwarp();
    }
    const SegDev &sg = p.segs[cur.seg];
    const DomW dd = dw[sg.domain];
    const uint64_t win0 = have ? (g - sg.tile_base) * kT : 0;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = !(have && cur.ok) ? 0u : (left < (uint64_t)kT ? (uint32_t)left : (uint32_t)kT);

    TileEnd te{0u, 0u, 0u};
    if (nwin) {
      te = decode_tile(p, cur, nwin * kE, dd, smem_raw, stage, lane, w, n);
      if (te.bad && lane == 0) flag_bad(p.status, te.bad, sg.caller_index);
    }
    if (g + 1 < t1) {  // tile g + 1 starts where tile g ended
      nxt = next_ctx(p, g, s, cur, te);
      pn = fetch_pass0(p, nxt, lane, wbuf);
    }
    __syncwarp();

    const float *deq = reinterpret_cast<const float *>(smem_raw + dd.deq_off);
    uint8_t *const lev = (want_lev && nwin) ? p.levels + sg.level_offset + win0 * kE : nullptr;
    for (uint32_t w0 = 0; w0 < (uint32_t)kT; w0 += kStepWin) {
      const uint32_t a_set = a_tmem + (uint32_t)(k & 1) * a_cols<MODE>();
      const uint32_t wi = w0 + lane;
      float c[16];
      if (wi < nwin) {
        const uint4 sv = *reinterpret_cast<const uint4 *>(stage + wi * kE);
        window_coefs(sv, deq, dd.zmask, c);
        if (lev) put_levels(lev + wi * kE, sv);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) c[j] = 0.0f;
      }
      put_a_row<MODE>(a_set + lane_off, c);  // product k - 1 reads the other A set
      tmem_wait_st();
      if (k > 0) drain(prev);                // D is free for product k once every warp has read it
      tc_fence_before();
      if (wg_barrier_any(wg, timeout)) {
        stop = true;
        break;
      }
      tc_fence_after();
      if (wq == 0 && lane == 0) {
        issue_products<MODE>(a_set, smem_addr(b_base), d_tmem);
        mma_commit(smem_addr(mbar + wg));
      }
      StepOut cur_out{0, nullptr, 0, 0, 0};
      if (w0 < nwin) {
        const uint32_t m = nwin - w0;
        cur_out.nwin = m < (uint32_t)kStepWin ? m : (uint32_t)kStepWin;
        cur_out.out_row = (sg.out_offset >> 5) + win0 + w0;
        cur_out.dst = p.out + sg.out_offset + (win0 + w0) * kN;
        cur_out.left = sg.n_samples - (win0 + w0) * kN;
        cur_out.flags = (sg.out_aligned & 1u) | ((sg.out_aligned & 2u) && vec32_base ? 2u : 0u) |
                        (wp.out_tma && (sg.out_aligned & 4u) ? 4u : 0u);
      }
      prev = cur_out;
      ++k;
    }
    __syncwarp();  // the level bytes are rewritten by the next tile
  }
  if (!stop && !timeout && k > 0) drain(prev);
  if (stop || timeout) {
    // An expired wait leaves the product it waited for possibly still writing
    // D (no later product was issued: the warpgroup stops at the barrier that
    // follows).  Wait for its commit once more, bounded, before the tensor
    // memory is released; the phase of that commit is the one before `phase`.
    mbar_wait(smem_addr(mbar + wg), phase ^ 1u);
    if (lane == 0) atomicOr(&p.status->flags, kFlagTimeout);
  }
  if (tma_pending && lane == 0) tma_wait_all();

  // ---- release tensor memory (every warp has finished its tcgen05.ld)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

template <int MODE, int NWG>
void *tcptr() {
  if constexpr (NWG * wg_cols<MODE>() <= 512u)
    return reinterpret_cast<void *>(&k_decode_tc<MODE, NWG>);
  else
    return nullptr;
}

template <int MODE>
void *tcpick_mode(uint32_t nwg) {
  switch (nwg) {
    case 1: return tcptr<MODE, 1>();
    case 2: return tcptr<MODE, 2>();
    case 3: return tcptr<MODE, 3>();
    case 4: return tcptr<MODE, 4>();
    case 5: return tcptr<MODE, 5>();
    case 6: return MODE == FPTC_IDCT_TF32X3 ? nullptr : tcptr<MODE, 6>();
    case 7: return MODE == FPTC_IDCT_TF32X3 ? nullptr : tcptr<MODE, 7>();
    default: return nullptr;
  }
}

void *tcpick(uint32_t mode, uint32_t threads) {
  if (threads % 128 != 0) return nullptr;
  const uint32_t nwg = threads / 128;
  switch (mode) {
    case FPTC_IDCT_TF32: return tcpick_mode<FPTC_IDCT_TF32>(nwg);
    case FPTC_IDCT_TF32X3: return tcpick_mode<FPTC_IDCT_TF32X3>(nwg);
    case FPTC_IDCT_BF16X3: return tcpick_mode<FPTC_IDCT_BF16X3>(nwg);
    default: return nullptr;
  }
}

}  // namespace

uint32_t tc_tile_windows() { return kT; }

// Shared-memory layout of the tensor-core kernel; returns total bytes.
size_t tc_smem_layout(uint32_t mode, uint32_t threads, const uint32_t *lmax, uint32_t n_domains, WarpParams *wp,
                      TcParams *tp) {
  const uint32_t nwg = threads / 128, warps = threads / 32;
  size_t o = align16(sizeof(DomW) * (n_domains ? n_domains : 1));
  wp->n_domains = n_domains;
  for (uint32_t d = 0; d < n_domains && d < kWarpMaxDomains; ++d) {
    wp->lut_off[d] = (uint32_t)o;
    o += align16((size_t)2 << lmax[d]);
    wp->tab_off[d] = (uint32_t)o;
    o += kDeqBytes;
  }
  o = align16(o);
  wp->warp_off = (uint32_t)o;
  wp->warp_bytes = (uint32_t)kMiscBytes;
  wp->out_tma = 0;
  o += (size_t)warps * kMiscBytes;
  tp->b_off = (uint32_t)align16(o);
  o = tp->b_off + (mode == FPTC_IDCT_TF32X3 ? 4096u : 2048u);  // B: TF32, BF16 hi + lo, or TF32 big + small
  tp->a_off = 0;         // A lives in tensor memory
  tp->a_buf = 0;
  tp->misc_off = (uint32_t)align16(o);
  o = tp->misc_off + 8 * nwg + 16;
  tp->tiles_off = (uint32_t)align16(o);
  const uint32_t cols = (mode == FPTC_IDCT_TF32X3 ? 96u : 64u) * nwg;  // wg_cols per warpgroup
  if (cols > 512u) return ~size_t(0);                                   // does not fit tensor memory
  // staging tiles aligned up to 1024 bytes from a 16-byte aligned offset: at most 1008 bytes skipped
  return tp->tiles_off + 1008 + (size_t)warps * kOutTile;
}

cudaError_t tc_smem_config(uint32_t mode, uint32_t threads, size_t smem) {
  void *k = tcpick(mode, threads);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return set_dynamic_smem_limit(k, smem);
}

cudaError_t tc_attributes(uint32_t mode, uint32_t threads, cudaFuncAttributes *attr) {
  void *k = tcpick(mode, threads);
  if (!k) return cudaErrorInvalidValue;
  return cudaFuncGetAttributes(attr, k);
}

cudaError_t tc_occupancy(uint32_t mode, uint32_t threads, size_t smem, int *ctas_per_sm) {
  void *k = tcpick(mode, threads);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, (int)threads, smem);
}

cudaError_t launch_tc(const DecodeParams &p, const WarpParams &wp, const TcParams &tp, const CUtensorMap &out_map,
                      uint32_t mode, uint32_t threads, uint32_t grid, size_t smem, cudaStream_t stream) {
  if (p.tile_end <= p.tile_begin || grid == 0) return cudaSuccess;
  void *k = tcpick(mode, threads);
  if (!k) return cudaErrorInvalidValue;
  DecodeParams pp = p;
  WarpParams ww = wp;
  TcParams tt = tp;
  CUtensorMap mm = out_map;
  void *args[] = {&pp, &ww, &tt, &mm};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
