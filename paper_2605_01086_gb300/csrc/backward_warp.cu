// Adjoint of the lossy decode stage for the Table 1 shape (N = 32, E = 16), one
// window per lane, on the warp-tile machinery (warp_tile.cuh).
//
// For a loss L with dL/dx = g (Sec. 4.2.2 run backwards):
//   g_C[w][k] = sum_n g[wN + n] B[k][n]            (B[0][n] = 1/2; samples past S are 0)
//   dL/dA_z  = sum over bins k of zone z of g_C[w][k] * unit_z(level[w][k])
// because the reconstruction of zone z is A_z * unit_z(level).  g_C is the
// DCT-II of the window's 32 gradients truncated to 16 bins; it is evaluated by
// the even/odd split that mirrors the forward transform: with
// u[n] = g[n] + g[31-n], v[n] = g[n] - g[31-n] the odd bins are
// sum_n v[n] B[2j+1][n] and the even bins the same construction on u (twice
// more), 232 FP32 operations per window with compile-time cosines.
//
// Per tile of 128 windows (a warp's contiguous tile range): levels come from
// the saved level buffer (16 bytes per window) or are decoded again; the
// gradient rows of each 32-window step arrive by a TMA tensor load into the
// warp's shared tile (rows of 32 floats, 128-byte swizzle; the next step's
// load is in flight while the current one is used); steps that are not whole,
// or whose output rows are not 128-byte aligned, are read directly.  Per
// window the lane forms sum_k g_C[k] * (A_z unit_z(L)) from the dequantization
// rows, per zone, scales it by 1 / A_z and adds it to an FP64 accumulator; the
// warp reduces its accumulators (FP64) and adds them to grad_scale with one
// FP64 atomic per zone whenever its domain changes and at the end.
#include "dct32.cuh"
#include "warp_tile.cuh"

namespace fptc {
namespace {

using namespace wt;
using namespace dct32;

constexpr int kGxTile = kStepWin * kN * 4;  // bytes of one step's gradient rows

// TMA load of rows [row, row + 32) of the gradient into a shared tile; the
// mbarrier completes when the bytes have arrived.
__device__ __forceinline__ void tma_load_rows(const CUtensorMap *map, void *smem_tile, uint32_t mbar, int32_t row) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"((uint32_t)kGxTile)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(smem_tile)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(mbar)
      : "memory");
}

// Where a step's gradient rows are: TMA tile (with its buffer) or direct reads.
struct StepIn {
  uint64_t row;   // first output row of the step (TMA)
  uint32_t tma;   // 1: the rows come by TMA
  uint32_t buf;   // its tile buffer
};

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) k_backward_warp(const BackwardParams bp, const WarpParams wp,
                                                                 const __grid_constant__ CUtensorMap gx_map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DecodeParams &p = bp.d;
  const DomW *const dw = reinterpret_cast<const DomW *>(smem_raw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  load_domain_tables<WARPS * 32>(p, wp.n_domains, smem_raw);

  unsigned char *const wbase = smem_raw + wp.warp_off + warp * kMiscBytes;
  uint64_t *const wbuf = reinterpret_cast<uint64_t *>(wbase);
  uint8_t *const stage = wbase + kStageOff;
  uint64_t *const mbar = reinterpret_cast<uint64_t *>(smem_raw + wp.warp_off + WARPS * kMiscBytes) + 2 * warp;
  const uintptr_t tiles0 =
      (reinterpret_cast<uintptr_t>(smem_raw + wp.warp_off + WARPS * kMiscBytes + WARPS * 16) + 1023) &
      ~uintptr_t(1023);
  unsigned char *const gtile = reinterpret_cast<unsigned char *>(tiles0) + warp * 2 * kGxTile;
  if (lane == 0) {
    mbar_init(smem_addr(mbar), 1);
    mbar_init(smem_addr(mbar + 1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const bool redecode = bp.levels_in == nullptr;
  uint64_t tw0, tw1;
  unit_tiles(p, (uint64_t)blockIdx.x * WARPS + warp, (uint64_t)gridDim.x * WARPS, tw0, tw1);
  if (tw0 >= tw1) return;

  uint32_t s = find_segment(p.segs, p.seg_begin, p.seg_end, tw0);
  uint32_t pn = 0;
  Ctx nxt{0, 0, 0, s, 0};
  if (redecode) {  // where tile tw0 starts, then its first words
    nxt = first_ctx(p, s, tw0, lane);
    pn = fetch_pass0(p, nxt, lane, wbuf);
  }

  uint32_t phase[2] = {0u, 0u};
  uint32_t nload = 0;       // TMA loads issued (buffer = count & 1)
  uint32_t pend = 0;        // buffers with a load not yet waited for (bit b = buffer b)
  bool timeout = false;
  double acc0 = 0.0, acc1 = 0.0;
  uint32_t acc_dom = 0xFFFFFFFFu;
  auto flush = [&]() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
      acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
    }
    if (lane == 0 && acc_dom != 0xFFFFFFFFu) {
      if (acc0 != 0.0) atomicAdd(bp.grad_scale + acc_dom * 3 + 0, acc0);
      if (acc1 != 0.0) atomicAdd(bp.grad_scale + acc_dom * 3 + 1, acc1);
    }
    acc0 = acc1 = 0.0;
  };

  for (uint64_t g = tw0; g < tw1 && !timeout; ++g) {
    while (g >= p.segs[s].tile_base + p.segs[s].n_tiles) ++s;
    Ctx cur{0, 0, 0, s, 1};
    uint64_t w[kWPL] = {0, 0};
    uint32_t n[kWPL] = {0, 0};
    if (redecode) {
      cp_async_wait_all();
      __syncwarp();
      cur = nxt;
#pragma unroll
      for (int u = 0; u < kWPL; ++u) {
        w[u] = wbuf[kWPL * lane + u];
        n[u] = (pn >> (8 * u)) & 0xffu;
      }
      __syncwarp();
      if (!cur.ok && g + 1 < tw1) {  // skipped tile: the next one is located without it
        nxt = next_ctx(p, g, s, cur, TileEnd{0u, 0u, 0u});
        pn = fetch_pass0(p, nxt, lane, wbuf);
      }
    }
    const SegDev &sg = p.segs[s];
    if (!cur.ok) continue;  // a segment the index flagged (only when decoding again)
    const DomW dd = dw[sg.domain];
    if (sg.domain != acc_dom) {
      flush();
      acc_dom = sg.domain;
    }
    const uint64_t win0 = (g - sg.tile_base) * kT;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = left < (uint64_t)kT ? (uint32_t)left : (uint32_t)kT;
    const float *deq = reinterpret_cast<const float *>(smem_raw + dd.deq_off);
    const float a0 = p.scale ? p.scale[sg.domain * 3 + 0] : p.domains[sg.domain].scale[0];
    const float a1 = p.scale ? p.scale[sg.domain * 3 + 1] : p.domains[sg.domain].scale[1];
    const float inv0 = a0 > 1e-30f ? 1.0f / a0 : 0.0f, inv1 = a1 > 1e-30f ? 1.0f / a1 : 0.0f;
    const bool tma_seg = wp.out_tma && (sg.out_aligned & 4u);
    const float *gsrc = bp.grad_out + sg.out_offset;
    float *const gco = bp.grad_coeffs ? bp.grad_coeffs + sg.level_offset + win0 * kE : nullptr;

    // first step's gradient rows in flight before the decode
    auto step_in = [&](uint32_t w0) -> StepIn {
      StepIn si{0, 0, 0};
      if (w0 >= nwin) return si;
      si.row = (sg.out_offset >> 5) + win0 + w0;
      si.tma = tma_seg && w0 + kStepWin <= nwin && (win0 + w0 + kStepWin) * kN <= sg.n_samples;
      return si;
    };
    // a TMA step's load goes to the buffer after the previous load's
    auto issue = [&](StepIn &si) {
      if (!si.tma) return;
      si.buf = nload & 1u;
      ++nload;
      pend |= 1u << si.buf;
      if (lane == 0) tma_load_rows(&gx_map, gtile + si.buf * kGxTile, smem_addr(mbar + si.buf), (int32_t)si.row);
    };
    StepIn si = step_in(0);  // first step's gradient rows in flight during the decode
    issue(si);

    if (redecode) {
      const TileEnd te = decode_tile(p, cur, nwin * kE, dd, smem_raw, stage, lane, w, n);
      if (te.bad && lane == 0) flag_bad(p.status, te.bad, sg.caller_index);
      if (g + 1 < tw1) {  // tile g + 1 starts where tile g ended
        nxt = next_ctx(p, g, s, cur, te);
        pn = fetch_pass0(p, nxt, lane, wbuf);
      }
      __syncwarp();
    }

    for (uint32_t w0 = 0; w0 < nwin; w0 += kStepWin) {
      const StepIn sn = step_in(w0 + kStepWin);
      const uint32_t wi = w0 + lane;
      // this step's rows (the next step's load is issued first)
      StepIn sn2 = sn;
      issue(sn2);
      float gx[32];
      if (si.tma) {
        const bool late = !mbar_wait(smem_addr(mbar + si.buf), phase[si.buf]);
        if (__any_sync(0xffffffffu, late)) {  // the load stays pending: waited for again below
          timeout = true;
          break;
        }
        phase[si.buf] ^= 1u;
        pend &= ~(1u << si.buf);
        const unsigned char *row = gtile + si.buf * kGxTile + lane * (kN * 4);
        const uint32_t sx = lane & 7u;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 q = *reinterpret_cast<const float4 *>(row + ((c ^ sx) << 4));
          gx[4 * c] = q.x;
          gx[4 * c + 1] = q.y;
          gx[4 * c + 2] = q.z;
          gx[4 * c + 3] = q.w;
        }
      } else {
        const uint64_t s0 = (win0 + wi) * kN;
#pragma unroll
        for (int j = 0; j < 32; ++j) gx[j] = (wi < nwin && s0 + j < sg.n_samples) ? __ldg(gsrc + s0 + j) : 0.0f;
      }
      if (wi < nwin) {
        uint4 sv;
        if (redecode) {
          sv = *reinterpret_cast<const uint4 *>(stage + wi * kE);
        } else {
          const uint8_t *ls = bp.levels_in + sg.level_offset + (win0 + wi) * kE;
          if ((reinterpret_cast<uintptr_t>(ls) & 15u) == 0) {
            sv = __ldg(reinterpret_cast<const uint4 *>(ls));
          } else {
            uint32_t q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int j = 0; j < 16; ++j) q[j >> 2] |= (uint32_t)__ldg(ls + j) << (8 * (j & 3));
            sv = make_uint4(q[0], q[1], q[2], q[3]);
          }
        }
        float gc[16];
        dct2_16(gx, gc);
        float c[16];
        window_coefs(sv, deq, dd.zmask, c);
        float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const uint32_t z = (dd.zmask >> (2 * k)) & 3u;
          if (z == 0) p0 = fmaf(gc[k], c[k], p0);
          if (z == 1) p1 = fmaf(gc[k], c[k], p1);
        }
        acc0 += (double)(p0 * inv0);
        acc1 += (double)(p1 * inv1);
        if (gco) {
          float *d = gco + wi * kE;
          if ((reinterpret_cast<uintptr_t>(d) & 31u) == 0) {
            const float lo[8] = {gc[0], gc[1], gc[2], gc[3], gc[4], gc[5], gc[6], gc[7]};
            const float hi[8] = {gc[8], gc[9], gc[10], gc[11], gc[12], gc[13], gc[14], gc[15]};
            st_cs_v8(d, lo);
            st_cs_v8(d + 8, hi);
          } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) d[k] = gc[k];
          }
        }
      }
      __syncwarp();  // every lane has read this step's tile before it is loaded again
      si = sn2;
    }
    __syncwarp();
  }
  // After an expired wait, up to two loads (the late one and the next step's)
  // may still be writing this warp's tiles: wait for them again, bounded, so
  // that no bulk copy into shared memory outlives the CTA.  Without a timeout
  // nothing is pending here (a tile's last step issues no further load).
  for (uint32_t b = 0; b < 2; ++b) {
    if (!(pend & (1u << b))) continue;
    mbar_wait(smem_addr(mbar + b), phase[b]);
  }
  flush();
  if (timeout && lane == 0) atomicOr(&p.status->flags, kFlagTimeout);
}

template <int WARPS>
void *bptr() {
  return reinterpret_cast<void *>(&k_backward_warp<WARPS>);
}
void *bpick(uint32_t threads) {
  switch (threads) {
    case 256: return bptr<8>();
    case 512: return bptr<16>();
    default: return nullptr;
  }
}

}  // namespace

size_t backward_warp_smem_layout(uint32_t threads, const uint32_t *lmax, uint32_t n_domains, WarpParams *wp) {
  const uint32_t warps = threads / 32;
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
  return o + (size_t)warps * kMiscBytes + (size_t)warps * 16 + 1023 + (size_t)warps * 2 * kGxTile;
}

cudaError_t backward_warp_smem_config(uint32_t threads, size_t smem) {
  void *k = bpick(threads);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return set_dynamic_smem_limit(k, smem);
}

cudaError_t launch_backward_warp(const BackwardParams &p, const WarpParams &wp, const CUtensorMap &gx_map,
                                 uint32_t threads, uint32_t grid, size_t smem, cudaStream_t stream) {
  if (p.d.tile_end <= p.d.tile_begin || grid == 0) return cudaSuccess;
  void *k = bpick(threads);
  if (!k) return cudaErrorInvalidValue;
  BackwardParams pp = p;
  WarpParams ww = wp;
  CUtensorMap mm = gx_map;
  void *args[] = {&pp, &ww, &mm};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
