// Tensor-core inverse transform for window shapes with E >= 32 (every domain
// of the plan the same N in {32, 64, 128} and E in {32, 64}, E <= N): the
// shapes where the FP32 transform costs E / 2 FMAs per sample and the
// contraction of Eq. 1's inverse
//      D[128 windows x N samples] = C[128 x E bins] * B[E x N],
//      B[k][n] = cos(pi/N (n + 1/2) k)  (B[0][n] = 1/2),
// is a real matrix product.  The structure is that of the N = 32, E = 16
// tensor-core kernel (decode_tc.cu): a warpgroup's four warps each decode a tile
// of T = 2048 / E windows (the warp-tile SymLen decode), then every 32-window
// step each lane dequantizes its window and writes its row of A into tensor
// memory (tcgen05.st), one thread issues the step's products (tcgen05.mma,
// M = 128, N samples, K = E, in the precision form's split) into the
// warpgroup's D, and the lanes read their window's N samples back 32 at a
// time (tcgen05.ld) and store them.  Two A sets per warpgroup (the next step's
// rows are written while the product runs) where four warpgroups still fit the
// 512 tensor-memory columns, else one (for more warpgroups).  A window's 32-sample chunk c
// leaves by a 3-D TMA tensor store (the output viewed as [windows][N / 32][32]
// floats: box 32 windows x 1 chunk x 32 floats, the staging tile's 128-byte
// swizzle) when the segment's output starts on a window boundary of that view
// and the step is whole, else by 32-byte, 16-byte or scalar stores.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc_ops.cuh"

namespace fptc {
namespace {

using namespace tcx;

// A set: columns of one step's A operand(s): TF32 E; TF32X3 big E + small E;
// BF16X3 hi E / 2 + lo E / 2 (two bf16 per column).
template <int MODE, int E>
__host__ __device__ constexpr uint32_t tcs_a_cols() {
  return MODE == FPTC_IDCT_TF32X3 ? 2u * E : (uint32_t)E;
}
// A sets per warpgroup: two (the next step's rows are written while the
// product runs) unless one set lets more warpgroups fit the 512 tensor-memory
// columns (then the rows are written after the previous product has
// finished); at most 5 warpgroups (registers and shared memory per warp).
constexpr uint32_t kTcsMaxWg = 5;
template <int MODE, int N, int E>
__host__ __device__ constexpr uint32_t tcs_nwg_for(uint32_t sets) {
  return 512u / ((uint32_t)N + sets * tcs_a_cols<MODE, E>()) < kTcsMaxWg
             ? 512u / ((uint32_t)N + sets * tcs_a_cols<MODE, E>())
             : kTcsMaxWg;
}
template <int MODE, int N, int E>
__host__ __device__ constexpr uint32_t tcs_asets() {
  return tcs_nwg_for<MODE, N, E>(2u) >= tcs_nwg_for<MODE, N, E>(1u) ? 2u : 1u;
}
template <int MODE, int N, int E>
__host__ __device__ constexpr uint32_t tcs_wg_cols() {
  return (uint32_t)N + tcs_asets<MODE, N, E>() * tcs_a_cols<MODE, E>();
}
template <int MODE, int N, int E>
__host__ __device__ constexpr uint32_t tcs_nwg() {
  return tcs_nwg_for<MODE, N, E>(tcs_asets<MODE, N, E>());
}
// B operand bytes (the small / lo part follows the big / hi one).
template <int MODE, int N, int E>
__host__ __device__ constexpr uint32_t tcs_b_bytes() {
  return MODE == FPTC_IDCT_TF32 ? N * E * 4u : MODE == FPTC_IDCT_TF32X3 ? 2u * N * E * 4u : 2u * N * E * 2u;
}

// B in shared memory, K-major, no swizzle (core matrices of 8 rows x 16 bytes):
// TF32 row n, bin k -> (n / 8) 32 E + (k / 4) 128 + (n % 8) 16 + (k % 4) 4 (LBO 128, SBO 32 E);
// BF16 row n, bin k -> (n / 8) 16 E + (k / 8) 128 + (n % 8) 16 + (k % 8) 2 (LBO 128, SBO 16 E).
template <int MODE, int N, int E>
__device__ __forceinline__ void tcs_fill_b(unsigned char *b_base, const float *bsrc, uint32_t t0, uint32_t stride) {
  for (uint32_t i = t0; i < (uint32_t)(N * E); i += stride) {
    const uint32_t n = i / E, k = i % E;
    const float b = __ldg(bsrc + k * N + n);
    if (MODE == FPTC_IDCT_BF16X3) {
      const __nv_bfloat16 bh = __float2bfloat16_rn(b);
      const __nv_bfloat16 bl = __float2bfloat16_rn(b - __bfloat162float(bh));
      const uint32_t o = (n >> 3) * 16u * E + (k >> 3) * 128u + (n & 7u) * 16u + (k & 7u) * 2u;
      *reinterpret_cast<__nv_bfloat16 *>(b_base + o) = bh;
      *reinterpret_cast<__nv_bfloat16 *>(b_base + N * E * 2u + o) = bl;
    } else {
      const float bb = tf32_round(b);
      const uint32_t o = (n >> 3) * 32u * E + (k >> 2) * 128u + (n & 7u) * 16u + (k & 3u) * 4u;
      *reinterpret_cast<float *>(b_base + o) = bb;
      if (MODE == FPTC_IDCT_TF32X3) *reinterpret_cast<float *>(b_base + N * E * 4u + o) = tf32_round(b - bb);
    }
  }
}

// Bins 16 q .. 16 q + 15 of this lane's row of the A operand(s): TF32 (and
// TF32X3's big part) at columns 16 q, TF32X3's small part at E + 16 q; BF16X3
// hi pairs at columns 8 q, lo pairs at E / 2 + 8 q.
template <int MODE, int E>
__device__ __forceinline__ void tcs_put_a16(uint32_t a, uint32_t q, const float (&c)[16]) {
  if (MODE == FPTC_IDCT_BF16X3) {
    uint32_t h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float x0 = c[2 * j], x1 = c[2 * j + 1];
      h[j] = pack_bf16(x0, x1);
      const float h0 = __uint_as_float(h[j] << 16), h1 = __uint_as_float(h[j] & 0xffff0000u);
      l[j] = pack_bf16(x0 - h0, x1 - h1);
    }
    tmem_st8(a + 8u * q, h);
    tmem_st8(a + E / 2 + 8u * q, l);
  } else {
    uint32_t big[16], sm[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (MODE == FPTC_IDCT_TF32X3) {
        // big = c with its 13 low mantissa bits cleared (a TF32 value), small = c - big exactly
        big[j] = __float_as_uint(c[j]) & 0xFFFFE000u;
        sm[j] = __float_as_uint(c[j] - __uint_as_float(big[j]));
      } else {
        big[j] = __float_as_uint(tf32_round(c[j]));
      }
    }
    tmem_st16(a + 16u * q, big);
    if (MODE == FPTC_IDCT_TF32X3) tmem_st16(a + E + 16u * q, sm);
  }
}

// The products of one step: A set at tensor-memory column a, B at shared address b, accumulator d.
template <int MODE, int N, int E>
__device__ __forceinline__ void tcs_issue(uint32_t a, uint32_t b, uint32_t d) {
  if (MODE == FPTC_IDCT_BF16X3) {
    constexpr uint32_t id = instr_desc(kFmtBF16, kRows, N);
    constexpr uint32_t sbo = 16u * E, lo = N * E * 2u;
#pragma unroll
    for (uint32_t h = 0; h < E / 16; ++h) {  // bins 16 h .. 16 h + 15
      mma_f16(d, a + 8 * h, smem_desc(b + 256 * h, 128, sbo), id, h > 0 ? 1u : 0u);  // hi * hi
      mma_f16(d, a + E / 2 + 8 * h, smem_desc(b + 256 * h, 128, sbo), id, 1);      // lo * hi
      mma_f16(d, a + 8 * h, smem_desc(b + lo + 256 * h, 128, sbo), id, 1);         // hi * lo
    }
  } else {
    constexpr uint32_t id = instr_desc(kFmtTF32, kRows, N);
    constexpr uint32_t sbo = 32u * E, sm = N * E * 4u;
#pragma unroll
    for (uint32_t h = 0; h < E / 8; ++h) {  // bins 8 h .. 8 h + 7
      mma_tf32(d, a + 8 * h, smem_desc(b + 256 * h, 128, sbo), id, h > 0 ? 1u : 0u);
      if (MODE == FPTC_IDCT_TF32X3) {
        mma_tf32(d, a + 8 * h, smem_desc(b + sm + 256 * h, 128, sbo), id, 1);  // big * small
        mma_tf32(d, a + E + 8 * h, smem_desc(b + 256 * h, 128, sbo), id, 1);   // small * big
      }
    }
  }
}

// 3-D TMA store of the staging tile: 32 windows' chunk `chunk` from window `win` on.
__device__ __forceinline__ void tma_store_chunk(const CUtensorMap *map, const void *tile, int32_t chunk, int32_t win) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(0), "r"(chunk), "r"(win), "r"(static_cast<uint32_t>(__cvta_generic_to_shared(tile)))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Output bookkeeping of a step whose product is in flight.
struct TcsOut {
  float *dst;         // first sample of window 0 of the step
  uint64_t left;      // samples of the segment from window 0 of the step on
  int64_t win;        // window index of window 0 in the output view (TMA), or -1
  uint32_t nwin;      // windows of the step (0..32)
  uint32_t flags;     // bit 0: 16-byte stores, bit 1: 32-byte stores
};

template <int MODE, int N, int E>
__global__ void __launch_bounds__(tcs_nwg<MODE, N, E>() * 128, 1)
    k_decode_tcs(const DecodeParams p, const WarpParams wp, const TcParams tp, const __grid_constant__ CUtensorMap out_map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NWG = (int)tcs_nwg<MODE, N, E>();
  constexpr int WARPS = NWG * 4;
  constexpr uint32_t T = kTS / E;  // windows per tile
  constexpr uint32_t CH = N / 32;  // 32-sample chunks per window
  const DomW *const dw = reinterpret_cast<const DomW *>(smem_raw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wg = warp >> 2, wq = warp & 3;

  // ---- tables, B operand(s), barriers, tensor memory
  load_domain_tables<WARPS * 32>(p, wp.n_domains, smem_raw);
  unsigned char *const b_base = smem_raw + tp.b_off;
  // every domain of the plan has this shape, so the same basis
  tcs_fill_b<MODE, N, E>(b_base, p.basis + p.domains[0].basis_offset, threadIdx.x, WARPS * 32);
  uint64_t *const mbar = reinterpret_cast<uint64_t *>(smem_raw + tp.misc_off);  // [NWG]
  uint32_t *const tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + tp.misc_off + 8 * NWG);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NWG; ++i) mbar_init(smem_addr(mbar + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr uint32_t kNeed = NWG * tcs_wg_cols<MODE, N, E>();
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
  const uint32_t d_tmem = tmem + wg * tcs_wg_cols<MODE, N, E>();  // this warpgroup's D, then its two A sets
  const uint32_t a_tmem = d_tmem + (uint32_t)N;
  const uint32_t lane_off = (wq * 32u) << 16;  // lanes 32 wq .. 32 wq + 31

  unsigned char *const wbase = smem_raw + wp.warp_off + warp * kMiscBytes;
  uint64_t *const wbuf = reinterpret_cast<uint64_t *>(wbase);
  uint8_t *const stage = wbase + kStageOff;
  const uintptr_t tiles0 = (reinterpret_cast<uintptr_t>(smem_raw + tp.tiles_off) + 1023) & ~uintptr_t(1023);
  unsigned char *const otile = reinterpret_cast<unsigned char *>(tiles0) + warp * kOutTile;
  unsigned char *const orow = otile + lane * 128u;
  const uint32_t sx = lane & 7u;
  const bool want_lev = p.levels != nullptr;
  const bool vec32_base = (reinterpret_cast<uintptr_t>(p.out) & 31u) == 0;

  // ---- this warp's tiles (an even split over all warps; the warpgroup runs
  // as many rounds as its longest range, a warp past its range contributing
  // zero rows)
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
  if (t0 < t1) {
    nxt = first_ctx(p, s, t0, lane, (uint64_t)T * E);
    pn = fetch_pass0(p, nxt, lane, wbuf);
  }

  uint32_t phase = 0u;
  bool timeout = false;
  bool stop = false;
  bool tma_pending = false;
  TcsOut prev{nullptr, 0, -1, 0, 0};
  uint64_t k = 0;  // steps issued by this warpgroup

  // Reads back the product in D (step k - 1), 32 samples per window at a time, and stores them.
  auto drain = [&](const TcsOut &o) {
    {
      const bool late = !mbar_wait(smem_addr(mbar + wg), phase);
      phase ^= 1u;
      timeout = timeout || __any_sync(0xffffffffu, late);
    }
    if (timeout) return;
    tc_fence_after();
    const bool tma = o.win >= 0 && o.nwin == 32u && (uint64_t)32u * N <= o.left;
#pragma unroll 1
    for (uint32_t c = 0; c < CH; ++c) {
      uint32_t v[32];
      tmem_ld32(d_tmem + 32u * c + lane_off, v);
      if (o.nwin == 0) continue;
      if (tma) {
        if (tma_pending) {
          if (lane == 0) tma_wait_read();
          __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<uint4 *>(orow + ((q ^ sx) << 4)) = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        fence_async_shared();
        __syncwarp();
        if (lane == 0) tma_store_chunk(&out_map, otile, (int32_t)c, (int32_t)o.win);
        tma_pending = true;
      } else if (lane < o.nwin) {
        const uint64_t s0 = (uint64_t)lane * N + 32u * c;  // first sample of this chunk from window 0 of the step
        float *const dst = o.dst + s0;
        if (s0 + 32 <= o.left && (o.flags & 2u)) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const float vv[8] = {__uint_as_float(v[8 * b]),     __uint_as_float(v[8 * b + 1]),
                                 __uint_as_float(v[8 * b + 2]), __uint_as_float(v[8 * b + 3]),
                                 __uint_as_float(v[8 * b + 4]), __uint_as_float(v[8 * b + 5]),
                                 __uint_as_float(v[8 * b + 6]), __uint_as_float(v[8 * b + 7])};
            st_cs_v8(dst + 8 * b, vv);
          }
        } else if (s0 + 32 <= o.left && (o.flags & 1u)) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            __stcs(reinterpret_cast<float4 *>(dst) + j,
                   make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                               __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3])));
        } else {
#pragma unroll
          for (int n = 0; n < 32; ++n)
            if (s0 + n < o.left) dst[n] = __uint_as_float(v[n]);
        }
      }
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
    const uint64_t win0 = have ? (g - sg.tile_base) * T : 0;
    const uint64_t left = sg.n_windows - win0;
    const uint32_t nwin = !(have && cur.ok) ? 0u : (left < (uint64_t)T ? (uint32_t)left : T);

    TileEnd te{0u, 0u, 0u};
    if (nwin) {
      te = decode_tile(p, cur, nwin * E, dd, smem_raw, stage, lane, w, n);
      if (te.bad && lane == 0) flag_bad(p.status, te.bad, sg.caller_index);
    }
    if (g + 1 < t1) {  // tile g + 1 starts where tile g ended
      nxt = next_ctx(p, g, s, cur, te);
      pn = fetch_pass0(p, nxt, lane, wbuf);
    }
    __syncwarp();

    const float *deq = reinterpret_cast<const float *>(smem_raw + dd.deq_off);
    const uint32_t B1 = p.domains[sg.domain].B1, B2 = p.domains[sg.domain].B2;
    uint8_t *const lev = (want_lev && nwin) ? p.levels + sg.level_offset + win0 * E : nullptr;
    // window index of the tile's first window in the output view [windows][N / 32][32]
    const int64_t vwin = (wp.out_tma && sg.out_offset % N == 0) ? (int64_t)(sg.out_offset / N + win0) : -1;
    for (uint32_t w0 = 0; w0 < T; w0 += 32) {
      constexpr uint32_t AS = tcs_asets<MODE, N, E>();
      const uint32_t a_set = a_tmem + (AS == 2u ? (uint32_t)(k & 1) * tcs_a_cols<MODE, E>() : 0u);
      const uint32_t wi = w0 + lane;
      // this lane's window: E coefficients dequantized and written 16 at a time
      auto put_row = [&]() {
#pragma unroll
        for (uint32_t q = 0; q < (uint32_t)E / 16; ++q) {
          float c[16];
          if (wi < nwin) {
            const uint4 u = reinterpret_cast<const uint4 *>(stage + wi * E)[q];
            const uint32_t sw[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const uint32_t kb = 16u * q + j;
              const uint32_t z = kb < B1 ? 0u : (kb < B2 ? 1u : 2u);
              c[j] = z < 2u ? deq[z * kZStride + ((sw[j >> 2] >> (8 * (j & 3))) & 0xffu)] : 0.0f;
            }
            if (lev) {
              uint8_t *dl = lev + wi * E + 16 * q;
              if ((reinterpret_cast<uintptr_t>(dl) & 15u) == 0) {
                *reinterpret_cast<uint4 *>(dl) = u;
              } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) dl[j] = (uint8_t)(sw[j >> 2] >> (8 * (j & 3)));
              }
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) c[j] = 0.0f;
          }
          tcs_put_a16<MODE, E>(a_set + lane_off, q, c);
        }
        tmem_wait_st();
      };
      if (AS == 2u) {
        put_row();                  // product k - 1 reads the other A set
        if (k > 0) drain(prev);     // D is free for product k once every warp has read it
      } else {
        if (k > 0) drain(prev);     // product k - 1 has read A and D is read back
        put_row();
      }
      tc_fence_before();
      if (wg_barrier_any(wg, timeout)) {
        stop = true;
        break;
      }
      tc_fence_after();
      if (wq == 0 && lane == 0) {
        tcs_issue<MODE, N, E>(a_set, smem_addr(b_base), d_tmem);
        mma_commit(smem_addr(mbar + wg));
      }
      TcsOut cur_out{nullptr, 0, -1, 0, 0};
      if (w0 < nwin) {
        const uint32_t m = nwin - w0;
        cur_out.nwin = m < 32u ? m : 32u;
        cur_out.dst = p.out + sg.out_offset + (win0 + w0) * N;
        cur_out.left = sg.n_samples - (win0 + w0) * N;
        cur_out.win = vwin >= 0 ? vwin + (int64_t)w0 : -1;
        cur_out.flags = (sg.out_aligned & 1u) | ((sg.out_aligned & 2u) && vec32_base ? 2u : 0u);
      }
      prev = cur_out;
      ++k;
    }
    __syncwarp();  // the level bytes are rewritten by the next tile
  }
  if (!stop && !timeout && k > 0) drain(prev);
  if (stop || timeout) {
    // the product waited for may still be writing D (no later one was issued):
    // wait for its commit once more, bounded, before tensor memory is released
    mbar_wait(smem_addr(mbar + wg), phase ^ 1u);
    if (lane == 0) atomicOr(&p.status->flags, kFlagTimeout);
  }
  if (tma_pending && lane == 0) tma_wait_all();

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

template <int MODE, int N, int E>
void *tcs_ptr() {
  return reinterpret_cast<void *>(&k_decode_tcs<MODE, N, E>);
}

template <int MODE>
void *tcs_pick_mode(uint32_t N, uint32_t E) {
  if (N == 32 && E == 32) return tcs_ptr<MODE, 32, 32>();
  if (N == 64 && E == 32) return tcs_ptr<MODE, 64, 32>();
  if (N == 128 && E == 32) return tcs_ptr<MODE, 128, 32>();
  if (N == 128 && E == 64) return tcs_ptr<MODE, 128, 64>();
  return nullptr;
}

void *tcs_pick(uint32_t mode, uint32_t N, uint32_t E) {
  switch (mode) {
    case FPTC_IDCT_TF32: return tcs_pick_mode<FPTC_IDCT_TF32>(N, E);
    case FPTC_IDCT_TF32X3: return tcs_pick_mode<FPTC_IDCT_TF32X3>(N, E);
    case FPTC_IDCT_BF16X3: return tcs_pick_mode<FPTC_IDCT_BF16X3>(N, E);
    default: return nullptr;
  }
}

template <int MODE>
uint32_t tcs_threads_mode(uint32_t N, uint32_t E) {
  if (N == 32 && E == 32) return tcs_nwg<MODE, 32, 32>() * 128u;
  if (N == 64 && E == 32) return tcs_nwg<MODE, 64, 32>() * 128u;
  if (N == 128 && E == 32) return tcs_nwg<MODE, 128, 32>() * 128u;
  if (N == 128 && E == 64) return tcs_nwg<MODE, 128, 64>() * 128u;
  return 0;
}

template <int MODE>
uint32_t tcs_b_bytes_mode(uint32_t N, uint32_t E) {
  if (N == 32 && E == 32) return tcs_b_bytes<MODE, 32, 32>();
  if (N == 64 && E == 32) return tcs_b_bytes<MODE, 64, 32>();
  if (N == 128 && E == 32) return tcs_b_bytes<MODE, 128, 32>();
  if (N == 128 && E == 64) return tcs_b_bytes<MODE, 128, 64>();
  return 0;
}

}  // namespace

bool tcs_supported(uint32_t N, uint32_t E) {
  return (N == 32 && E == 32) || (N == 64 && E == 32) || (N == 128 && E == 32) || (N == 128 && E == 64);
}

uint32_t tcs_tile_windows(uint32_t E) { return E ? (uint32_t)kTS / E : 0u; }

uint32_t tcs_threads(uint32_t mode, uint32_t N, uint32_t E) {
  switch (mode) {
    case FPTC_IDCT_TF32: return tcs_threads_mode<FPTC_IDCT_TF32>(N, E);
    case FPTC_IDCT_TF32X3: return tcs_threads_mode<FPTC_IDCT_TF32X3>(N, E);
    case FPTC_IDCT_BF16X3: return tcs_threads_mode<FPTC_IDCT_BF16X3>(N, E);
    default: return 0;
  }
}

// Shared-memory layout of the shape tensor-core kernel; returns total bytes
// (~0 for a shape or form it does not serve).
size_t tcs_smem_layout(uint32_t mode, uint32_t N, uint32_t E, const uint32_t *lmax, uint32_t n_domains,
                       WarpParams *wp, TcParams *tp) {
  const uint32_t threads = tcs_threads(mode, N, E);
  if (!threads || !tcs_supported(N, E)) return ~size_t(0);
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
  const uint32_t bb = mode == FPTC_IDCT_TF32 ? tcs_b_bytes_mode<FPTC_IDCT_TF32>(N, E)
                      : mode == FPTC_IDCT_TF32X3 ? tcs_b_bytes_mode<FPTC_IDCT_TF32X3>(N, E)
                                                 : tcs_b_bytes_mode<FPTC_IDCT_BF16X3>(N, E);
  o = tp->b_off + bb;
  tp->a_off = 0;  // A lives in tensor memory
  tp->a_buf = 0;
  tp->misc_off = (uint32_t)align16(o);
  o = tp->misc_off + 8 * nwg + 16;
  tp->tiles_off = (uint32_t)align16(o);
  return tp->tiles_off + 1023 + (size_t)warps * kOutTile;
}

cudaError_t tcs_smem_config(uint32_t mode, uint32_t N, uint32_t E, size_t smem) {
  void *k = tcs_pick(mode, N, E);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return set_dynamic_smem_limit(k, smem);
}

cudaError_t tcs_occupancy(uint32_t mode, uint32_t N, uint32_t E, size_t smem, int *ctas_per_sm) {
  void *k = tcs_pick(mode, N, E);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, (int)tcs_threads(mode, N, E), smem);
}

// The output as [windows][N / 32][32] floats for the 3-D TMA stores (box 32
// floats x 1 chunk x 32 windows, 128-byte swizzle).  False when it cannot be
// described (then every step stores with the lanes).
bool encode_out_map3(CUtensorMap *map, float *out, uint64_t extent, uint32_t N) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  const uint64_t wins = N ? extent / N : 0;
  if (!encode || !out || N < 32 || N % 32 || (reinterpret_cast<uintptr_t>(out) & 15u) || wins == 0 ||
      wins > 0x7FFFFFFFull)
    return false;
  const cuuint64_t dims[3] = {32, (cuuint64_t)(N / 32), (cuuint64_t)wins};
  const cuuint64_t strides[2] = {128, (cuuint64_t)N * 4};
  const cuuint32_t box[3] = {32, 1, 32};
  const cuuint32_t estride[3] = {1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, out, dims, strides, box, estride,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_tcs(const DecodeParams &p, const WarpParams &wp, const TcParams &tp, const CUtensorMap &out_map,
                       uint32_t mode, uint32_t N, uint32_t E, uint32_t grid, size_t smem, cudaStream_t stream) {
  if (p.tile_end <= p.tile_begin || grid == 0) return cudaSuccess;
  void *k = tcs_pick(mode, N, E);
  if (!k) return cudaErrorInvalidValue;
  DecodeParams pp = p;
  WarpParams ww = wp;
  TcParams tt = tp;
  CUtensorMap mm = out_map;
  void *args[] = {&pp, &ww, &tt, &mm};
  return cudaLaunchKernel(k, dim3(grid), dim3(tcs_threads(mode, N, E)), args, smem, stream);
}

}  // namespace fptc
