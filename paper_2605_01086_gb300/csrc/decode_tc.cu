// Fused decode with the inverse DCT on the 5th-generation tensor cores
// (tcgen05, accumulator in tensor memory), for the Table 1 shape N = 32, E = 16.
//
// A warpgroup (4 warps) works on 128 windows at a time: warp w Huffman-decodes
// and dequantizes one tile of 32 windows (Sec. 4.2.1 / 4.2.2, same decode as
// the other kernels) into a per-warp coefficient buffer, then repacks its 32
// rows into the operand layout of the matrix multiply
//      D[128 windows x 32 samples] = C[128 x 16 bins] * B[16 x 32]
// with B[k][n] = cos(pi/N (n + 1/2) k) (B[0][n] = 1/2), the inverse of Eq. 1.
// One thread issues the tcgen05.mma instructions (M = 128, N = 32) with A and
// B in shared memory and D in tensor memory; tcgen05.commit signals an
// mbarrier; then every warp reads its 32 rows of D with tcgen05.ld (lane i of
// warp w holds row 32w + i = one window) and stores the window's 32 samples.
//
// A kernel that uses tensor memory runs one CTA per SM (the occupancy the CUDA
// runtime reports for it is 1), so all warpgroups of an SM live in one CTA.
//
// Precision forms (the integer decode is exact in every form):
//   TF32    one product, operands rounded to TF32 (10-bit mantissa);
//   TF32X3  C = C_big + C_small, B = B_big + B_small (TF32 each), three
//           products C_big B_big + C_big B_small + C_small B_big;
//   BF16X3  the same split with BF16 halves, C_hi B_hi + C_lo B_hi + C_hi B_lo.
// All accumulate in FP32.
//
// Operand layout: K-major, no swizzle.  A core matrix is 8 rows x 16 bytes
// stored contiguously; LBO = byte distance between core matrices adjacent in K,
// SBO = between core matrices adjacent in M (or N).  Every wait on the mbarrier
// is bounded; on timeout the kernel flags FPTC_FLAG_TIMEOUT and stops.
#include <cuda_bf16.h>

#include "device_util.cuh"

namespace fptc {
namespace {

constexpr int kN = 32;
constexpr int kE = 16;
constexpr int kT = 32;          // windows per warp tile
constexpr int kTS = kT * kE;    // symbols per warp tile
constexpr int kGuard = 64;
constexpr int kZStride = 257;
constexpr int kRows = 128;      // windows per warpgroup tile (MMA M)
constexpr uint32_t kWaitLimit = 1u << 26;

// ---- small PTX wrappers -----------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// OR of a predicate over the 128 threads of named barrier ID (and a barrier).
// The id is a compile-time constant: a run-time id makes the compiler reserve
// every hardware barrier of the SM for one CTA.
template <int ID>
__device__ __forceinline__ bool bar_any_c(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, 128, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(ID)
      : "memory");
  return r != 0;
}

// Barrier over the 128 threads of warpgroup wg (ids 1..4), returning the OR of v.
__device__ __forceinline__ bool wg_barrier_any(uint32_t wg, bool v) {
  switch (wg) {
    case 0: return bar_any_c<1>(v);
    case 1: return bar_any_c<2>(v);
    case 2: return bar_any_c<3>(v);
    default: return bar_any_c<4>(v);
  }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 at bits 0-13, LBO >> 4
// at 16-29, SBO >> 4 at 32-45, descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor: D format F32 (bits 4-5 = 1), A/B format at bits 7-9 /
// 10-12, K-major A and B, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_format, uint32_t m, uint32_t n) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
constexpr uint32_t kFmtBF16 = 1, kFmtTF32 = 2;

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---- operand layouts ---------------------------------------------------------

// TF32 (4 bytes): row r, bin k -> (r/8)*512 + (k/4)*128 + (r%8)*16 + (k%4)*4; LBO 128, SBO 512.
// BF16 (2 bytes): row r, bin k -> (r/8)*256 + (k/8)*128 + (r%8)*16 + (k%8)*2; LBO 128, SBO 256.
__device__ __forceinline__ uint32_t off_tf32_chunk(uint32_t r, uint32_t j) {
  return (r >> 3) * 512u + j * 128u + (r & 7u) * 16u;
}
__device__ __forceinline__ uint32_t off_bf16_chunk(uint32_t r, uint32_t j) {
  return (r >> 3) * 256u + j * 128u + (r & 7u) * 16u;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// ---- decode (same SymLen decode as the other kernels) --------------------------

struct TcTile {
  uint64_t fw;
  uint32_t nw;
  uint32_t skip;
};

__device__ __forceinline__ TcTile tc_ctx(const SegDev &sg, uint64_t tin, const TileRec &r, const TileRec &rn) {
  TcTile c;
  c.fw = r.first_word;
  c.skip = r.skip;
  uint64_t lw;
  if (tin + 1 < sg.n_tiles)
    lw = rn.first_word - (rn.skip == 0 ? 1u : 0u);
  else
    lw = sg.word_offset + sg.n_words - 1;
  c.nw = lw >= c.fw ? (uint32_t)(lw - c.fw + 1) : 0u;
  return c;
}

template <int WPT>
__device__ __forceinline__ unsigned tc_decode(const uint64_t (&wd)[WPT], const uint32_t (&sl)[WPT], int32_t q0,
                                              int32_t tsyms, const uint16_t *__restrict__ lut, uint32_t shift,
                                              uint32_t zmask, const float *__restrict__ deq,
                                              float *__restrict__ coef, uint8_t *__restrict__ lev, bool checked,
                                              bool write_lev) {
  uint32_t hi[WPT], lo[WPT], cnt[WPT], used[WPT];
  int32_t q[WPT];
  uint32_t maxc = 0;
  int32_t qq = q0;
#pragma unroll
  for (int u = 0; u < WPT; ++u) {
    hi[u] = (uint32_t)(wd[u] >> 32);
    lo[u] = (uint32_t)wd[u];
    q[u] = qq;
    const int32_t room = tsyms - qq;
    cnt[u] = room <= 0 ? 0u : min(sl[u], (uint32_t)room);
    qq += (int32_t)sl[u];
    used[u] = 0;
    maxc = max(maxc, cnt[u]);
  }
  bool bad = false;
  for (uint32_t j = 0; j < maxc; ++j) {
#pragma unroll
    for (int u = 0; u < WPT; ++u) {
      if (j < cnt[u]) {
        const uint32_t e = lut[hi[u] >> shift];
        const uint32_t len = e >> 8;
        if (checked) bad |= len == 0;
        hi[u] = __funnelshift_l(lo[u], hi[u], len);
        lo[u] <<= len;
        used[u] += len;
        const uint32_t sym = e & 0xffu;
        const uint32_t z = (zmask >> (2u * (uint32_t)(q[u] & (kE - 1)))) & 3u;
        coef[q[u]] = deq[z * kZStride + sym];
        if (write_lev) lev[q[u]] = (uint8_t)sym;
        ++q[u];
      }
    }
  }
  unsigned err = bad ? kFlagInvalidCode : 0u;
#pragma unroll
  for (int u = 0; u < WPT; ++u)
    if (used[u] > 64u) err |= kFlagBitOverrun;
  return err;
}

struct DomTc {
  uint32_t lut_off;
  uint32_t tab_off;
  uint32_t shift;
  uint32_t zmask;
  uint32_t complete;
  uint32_t pad[3];
};

// Where warp w's current tile writes: valid flag, segment fields for the epilogue.
struct EpiCtx {
  float *out;        // segment output base
  uint64_t s0;       // first sample of the tile in the segment
  uint64_t S;        // segment length
  uint32_t nwin;     // windows in the tile (0 = nothing to store)
  uint32_t aligned;
};

template <int NWG>
constexpr int tc_min_blocks() {
  return NWG >= 4 ? 1 : 2;
}

template <int MODE, int NWG>
__global__ void __launch_bounds__(NWG * 128, tc_min_blocks<NWG>()) k_decode_tc(const DecodeParams p, const TcParams tp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int WPT = 2;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wg = warp >> 2, wq = warp & 3;  // warpgroup, warp within it

  // ---- layout (bytes; host computes the same in tc_smem_layout)
  unsigned char *const a_base = smem_raw + tp.a_off + wg * tp.a_bytes;          // per warpgroup A operand(s)
  float *const coef = reinterpret_cast<float *>(smem_raw + tp.coef_off + warp * tp.coef_bytes) + kGuard;
  uint8_t *const lev = smem_raw + tp.coef_off + warp * tp.coef_bytes + (kGuard + kTS) * 4 + kGuard;
  unsigned char *const b_base = smem_raw + tp.b_off;                             // B operand(s)
  uint64_t *const mbar = reinterpret_cast<uint64_t *>(smem_raw + tp.misc_off);   // [NWG][2]
  uint32_t *const tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + tp.misc_off + 16 * NWG);
  DomTc *const ds = reinterpret_cast<DomTc *>(smem_raw + tp.dom_off);

  const uint64_t n_all = p.tile_end - p.tile_begin;
  const uint64_t t0 = p.tile_begin + n_all * blockIdx.x / gridDim.x;
  const uint64_t t1 = p.tile_begin + n_all * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;  // whole CTA: no tensor memory taken

  // ---- domain tables, B operand, barriers, tensor memory
  uint32_t off = tp.tab_first;
  for (uint32_t d = 0; d < tp.n_domains; ++d) {
    const DomainDev &dm = p.domains[d];
    const uint32_t lut_off = off;
    const uint32_t tab_off = lut_off + (uint32_t)align16((size_t)2 << dm.lmax);
    off = tab_off + (uint32_t)align16(3u * kZStride * 4);
    if (threadIdx.x == 0) {
      DomTc x;
      x.lut_off = lut_off;
      x.tab_off = tab_off;
      x.shift = 32u - dm.lmax;
      uint32_t zm = 0;
      for (uint32_t k = 0; k < kE; ++k) zm |= (k < dm.B1 ? 0u : (k < dm.B2 ? 1u : 2u)) << (2 * k);
      x.zmask = zm;
      x.complete = dm.complete;
      x.pad[0] = x.pad[1] = x.pad[2] = 0;
      ds[d] = x;
    }
    load_lut<NWG * 128>(reinterpret_cast<uint16_t *>(smem_raw + lut_off), p.luts + dm.lut_offset, 1u << dm.lmax);
    float a0 = p.scale ? p.scale[d * 3 + 0] : dm.scale[0];
    float a1 = p.scale ? p.scale[d * 3 + 1] : dm.scale[1];
    a0 = a0 > 1e-30f ? a0 : 0.0f;
    a1 = a1 > 1e-30f ? a1 : 0.0f;
    float *deq = reinterpret_cast<float *>(smem_raw + tab_off);
    for (uint32_t i = threadIdx.x; i < 3u * kZStride; i += NWG * 128) {
      const uint32_t z = i / kZStride, L = i - z * kZStride;
      deq[i] = (L < 256u && z < 2u) ? (z == 0 ? a0 : a1) * dm.unit[z][L] : 0.0f;
    }
  }
  {
    // B operand: row n (sample), bin k; every domain of this kernel shares it
    const float *bsrc = p.basis + p.domains[0].basis_offset;  // [k][n]
    for (uint32_t i = threadIdx.x; i < kN * kE; i += NWG * 128) {
      const uint32_t n = i / kE, k = i % kE;
      const float b = __ldg(bsrc + k * kN + n);
      if (MODE == FPTC_IDCT_BF16X3) {
        const __nv_bfloat16 bh = __float2bfloat16_rn(b);
        const __nv_bfloat16 bl = __float2bfloat16_rn(b - __bfloat162float(bh));
        const uint32_t o = (n >> 3) * 256u + (k >> 3) * 128u + (n & 7u) * 16u + (k & 7u) * 2u;
        *reinterpret_cast<__nv_bfloat16 *>(b_base + o) = bh;
        *reinterpret_cast<__nv_bfloat16 *>(b_base + 1024 + o) = bl;
      } else {
        const float bb = tf32_round(b);
        const uint32_t o = (n >> 3) * 512u + (k >> 2) * 128u + (n & 7u) * 16u + (k & 3u) * 4u;
        *reinterpret_cast<float *>(b_base + o) = bb;
        if (MODE == FPTC_IDCT_TF32X3) *reinterpret_cast<float *>(b_base + 2048 + o) = tf32_round(b - bb);
      }
    }
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * NWG; ++i) mbar_init(smem_u32(mbar + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr uint32_t kCols = NWG == 1 ? 64u : (NWG == 2 ? 128u : 256u);  // two 32-column D per warpgroup
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async_smem();  // B operand written by threads, read by the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t d_tmem = tmem + wg * 64u;                 // this warpgroup's two 32-column D buffers
  const uint32_t my_tmem = d_tmem + ((wq * 32u) << 16);    // lanes 32 wq .. 32 wq + 31

  const bool want_lev = p.levels != nullptr;
  uint32_t phase[2] = {0u, 0u};
  bool timeout = false;

  // Warpgroup tile k = 4 consecutive warp tiles t0 + 4 (wg + k NWG) + wq.  The
  // pipeline: decode tile k+1 into A[(k+1) & 1] while the products of tile k
  // run on the tensor core into D[k & 1]; then wait, store tile k, barrier,
  // issue tile k+1.
  auto gbase_of = [&](uint64_t k) -> uint64_t { return t0 + 4 * (wg + k * NWG); };
  EpiCtx ep0{nullptr, 0, 0, 0, 0}, ep1{nullptr, 0, 0, 0, 0};  // per A/D buffer (no dynamic index: registers)

  // Per-warp prefetch state: the segment cursor, the context and words of the
  // next tile this warp decodes, the context of the one after (records only).
  uint32_t s_cur = find_segment(p.segs, p.seg_begin, p.seg_end, min(gbase_of(0) + wq, t1 - 1));
  bool bad_cur = true, bad_nxt = true;
  uint32_t s_nxt = s_cur;
  TcTile cx_cur{0, 0, 0}, cx_nxt{0, 0, 0};
  uint64_t pw[WPT];
  uint32_t psl[WPT];
  // context of warp tile g (segment cursor s advanced to it); records only
  auto ctx_of = [&](uint64_t g, uint32_t &s, bool &bad, TcTile &cx) {
    bad = true;
    if (g >= t1) return;
    while (g >= p.segs[s].tile_base + p.segs[s].n_tiles) ++s;
    bad = p.seg_bad[s] != 0;
    if (bad) return;
    const SegDev &sg = p.segs[s];
    const uint64_t tin = g - sg.tile_base;
    TileRec rn{0, 0, 0};
    if (tin + 1 < sg.n_tiles) rn = p.tiles[g + 1];
    cx = tc_ctx(sg, tin, p.tiles[g], rn);
  };
  auto load_words = [&](bool bad, const TcTile &cx) {
#pragma unroll
    for (int u = 0; u < WPT; ++u) {
      const uint32_t i = lane * WPT + u;
      const bool in = !bad && i < cx.nw;
      psl[u] = in ? (uint32_t)__ldg(p.symlen + cx.fw + i) : 0u;
      pw[u] = in ? __ldg(p.words + cx.fw + i) : 0ull;
    }
  };
  ctx_of(gbase_of(0) + wq, s_cur, bad_cur, cx_cur);
  load_words(bad_cur, cx_cur);
  s_nxt = s_cur;
  ctx_of(gbase_of(1) + wq, s_nxt, bad_nxt, cx_nxt);

  // decode + repack of warpgroup tile k (whose context and words are loaded)
  // into A buffer `buf`; then start the loads of tile k+1 and the records of
  // tile k+2
  auto produce = [&](uint64_t k, uint32_t buf) {
    const uint64_t g = gbase_of(k) + wq;
    EpiCtx e{nullptr, 0, 0, 0, 0};
    unsigned err = 0;
    uint64_t wd0[WPT];
    uint32_t sl0[WPT];
#pragma unroll
    for (int u = 0; u < WPT; ++u) {
      wd0[u] = pw[u];
      sl0[u] = psl[u];
    }
    const bool bad = bad_cur;
    const uint32_t s = s_cur;
    const TcTile cx = cx_cur;
    // rotate the prefetch: words of tile k+1 now, records of tile k+2
    s_cur = s_nxt;
    bad_cur = bad_nxt;
    cx_cur = cx_nxt;
    load_words(bad_cur, cx_cur);
    s_nxt = s_cur;
    ctx_of(gbase_of(k + 2) + wq, s_nxt, bad_nxt, cx_nxt);
    if (g < t1) {
      if (!bad) {
        const SegDev &sg = p.segs[s];
        const DomTc dd = ds[sg.domain];
        const uint64_t tin = g - sg.tile_base;
        const uint64_t win0 = tin * kT;
        const uint64_t left = sg.n_windows - win0;
        const uint32_t nwin = left < (uint64_t)kT ? (uint32_t)left : (uint32_t)kT;
        const int32_t tsyms = (int32_t)(nwin * kE);
        const uint16_t *lut = reinterpret_cast<const uint16_t *>(smem_raw + dd.lut_off);
        const float *deq = reinterpret_cast<const float *>(smem_raw + dd.tab_off);
        int32_t base = -(int32_t)cx.skip;
        for (uint32_t c0 = 0; c0 < cx.nw; c0 += 32 * WPT) {
          uint64_t wd[WPT];
          uint32_t sl[WPT];
          uint32_t tsum = 0;
#pragma unroll
          for (int u = 0; u < WPT; ++u) {
            if (c0 == 0) {
              wd[u] = wd0[u];
              sl[u] = sl0[u];
            } else {
              const uint32_t i = c0 + lane * WPT + u;
              const bool in = i < cx.nw;
              sl[u] = in ? (uint32_t)__ldg(p.symlen + cx.fw + i) : 0u;
              wd[u] = in ? __ldg(p.words + cx.fw + i) : 0ull;
            }
            tsum += sl[u];
          }
          uint32_t x = tsum;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
          }
          const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
          if (tsum)
            err |= tc_decode<WPT>(wd, sl, base + (int32_t)(x - tsum), tsyms, lut, dd.shift, dd.zmask, deq, coef,
                                  lev, dd.complete == 0, want_lev);
          base += (int32_t)total;
          if (base >= tsyms) break;
        }
        if (err) flag_bad(p.status, err, sg.caller_index);
        __syncwarp();
        if (want_lev) {
          uint8_t *dst = p.levels + sg.level_offset + win0 * kE;
          for (int32_t i = lane; i < tsyms; i += 32) dst[i] = lev[i];
        }
        e.out = p.out + sg.out_offset;
        e.s0 = win0 * kN;
        e.S = sg.n_samples;
        e.nwin = nwin;
        e.aligned = sg.out_aligned;
      }
    }
    // repack: lane i moves window i of this warp's tile into the A operand(s)
    // (rows of windows that are not in the tile keep stale values; their D rows
    // are never stored)
    unsigned char *const a = a_base + buf * tp.a_buf;
    if (lane < e.nwin) {
      const uint32_t r = wq * 32u + lane;
      const float4 *src = reinterpret_cast<const float4 *>(coef + lane * kE);
      float4 c[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) c[j] = src[j];
      if (MODE == FPTC_IDCT_BF16X3) {
        uint32_t h[8], l[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float v[4] = {c[j].x, c[j].y, c[j].z, c[j].w};
          float hv[4], lv[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            hv[t] = __bfloat162float(__float2bfloat16_rn(v[t]));
            lv[t] = v[t] - hv[t];
          }
          h[2 * j] = pack_bf16(hv[0], hv[1]);
          h[2 * j + 1] = pack_bf16(hv[2], hv[3]);
          l[2 * j] = pack_bf16(lv[0], lv[1]);
          l[2 * j + 1] = pack_bf16(lv[2], lv[3]);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          *reinterpret_cast<uint4 *>(a + off_bf16_chunk(r, j)) =
              make_uint4(h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]);
          *reinterpret_cast<uint4 *>(a + 4096 + off_bf16_chunk(r, j)) =
              make_uint4(l[4 * j], l[4 * j + 1], l[4 * j + 2], l[4 * j + 3]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 big = make_float4(tf32_round(c[j].x), tf32_round(c[j].y), tf32_round(c[j].z),
                                         tf32_round(c[j].w));
          *reinterpret_cast<float4 *>(a + off_tf32_chunk(r, j)) = big;
          if (MODE == FPTC_IDCT_TF32X3) {
            const float4 sm = make_float4(tf32_round(c[j].x - big.x), tf32_round(c[j].y - big.y),
                                          tf32_round(c[j].z - big.z), tf32_round(c[j].w - big.w));
            *reinterpret_cast<float4 *>(a + 8192 + off_tf32_chunk(r, j)) = sm;
          }
        }
      }
    }
    fence_proxy_async_smem();
    if (buf)
      ep1 = e;
    else
      ep0 = e;
  };

  // one thread issues the products of A buffer `buf` into D buffer `buf`
  auto issue = [&](uint32_t buf) {
    if (wq == 0 && lane == 0) {
      tc_fence_after();
      const uint32_t a = smem_u32(a_base + buf * tp.a_buf), b = smem_u32(b_base);
      const uint32_t d = d_tmem + buf * 32u;
      if (MODE == FPTC_IDCT_BF16X3) {
        constexpr uint32_t id = instr_desc(kFmtBF16, kRows, kN);
        mma_f16(d, smem_desc(a, 128, 256), smem_desc(b, 128, 256), id, 0);          // hi * hi
        mma_f16(d, smem_desc(a + 4096, 128, 256), smem_desc(b, 128, 256), id, 1);   // lo * hi
        mma_f16(d, smem_desc(a, 128, 256), smem_desc(b + 1024, 128, 256), id, 1);   // hi * lo
      } else {
        constexpr uint32_t id = instr_desc(kFmtTF32, kRows, kN);
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h) {  // bins 0..7, 8..15
          mma_tf32(d, smem_desc(a + 256 * h, 128, 512), smem_desc(b + 256 * h, 128, 512), id, h);
          if (MODE == FPTC_IDCT_TF32X3) {
            mma_tf32(d, smem_desc(a + 256 * h, 128, 512), smem_desc(b + 2048 + 256 * h, 128, 512), id, 1);
            mma_tf32(d, smem_desc(a + 8192 + 256 * h, 128, 512), smem_desc(b + 256 * h, 128, 512), id, 1);
          }
        }
      }
      mma_commit(smem_u32(mbar + 2 * wg + buf));
    }
  };

  if (gbase_of(0) < t1) {
    produce(0, 0);
    tc_fence_before();
    wg_barrier_any(wg, false);
    issue(0);
    for (uint64_t k = 0;; ++k) {
      const uint32_t buf = (uint32_t)(k & 1);
      const bool has_next = gbase_of(k + 1) < t1;  // uniform over the warpgroup
      if (has_next) produce(k + 1, buf ^ 1u);
      // wait for tile k's products (bounded)
      {
        uint32_t it = 0;
        while (!mbar_try_wait(smem_u32(mbar + 2 * wg + buf), phase[buf])) {
          if (++it >= kWaitLimit) {
            timeout = true;
            break;
          }
        }
        phase[buf] ^= 1u;
      }
      if (!timeout) {
        tc_fence_after();
        uint32_t v[32];
        tmem_ld32(my_tmem + buf * 32u, v);
        const EpiCtx e = buf ? ep1 : ep0;
        if (lane < e.nwin) {
          const uint64_t s0 = e.s0 + (uint64_t)lane * kN;
          float *dst = e.out + s0;
          if (s0 + kN <= e.S && e.aligned) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcs(reinterpret_cast<float4 *>(dst) + j,
                     make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                 __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3])));
          } else {
#pragma unroll
            for (int n = 0; n < kN; ++n)
              if (s0 + n < e.S) dst[n] = __uint_as_float(v[n]);
          }
        }
      }
      // every warp of the warpgroup: tile k+1 repacked, tile k read; one
      // decision about a timeout for all of them
      tc_fence_before();
      if (wg_barrier_any(wg, timeout)) {
        if (threadIdx.x % 128 == 0) atomicOr(&p.status->flags, kFlagTimeout);
        break;
      }
      if (!has_next) break;
      issue(buf ^ 1u);
    }
  }
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
  return reinterpret_cast<void *>(&k_decode_tc<MODE, NWG>);
}

void *tcpick(uint32_t mode, uint32_t threads) {
  const uint32_t nwg = threads / 128;
  switch (mode) {
    case FPTC_IDCT_TF32:
      return nwg == 1 ? tcptr<FPTC_IDCT_TF32, 1>() : (nwg == 2 ? tcptr<FPTC_IDCT_TF32, 2>() : (nwg == 4 ? tcptr<FPTC_IDCT_TF32, 4>() : nullptr));
    case FPTC_IDCT_TF32X3:
      return nwg == 1 ? tcptr<FPTC_IDCT_TF32X3, 1>() : (nwg == 2 ? tcptr<FPTC_IDCT_TF32X3, 2>() : (nwg == 4 ? tcptr<FPTC_IDCT_TF32X3, 4>() : nullptr));
    case FPTC_IDCT_BF16X3:
      return nwg == 1 ? tcptr<FPTC_IDCT_BF16X3, 1>() : (nwg == 2 ? tcptr<FPTC_IDCT_BF16X3, 2>() : (nwg == 4 ? tcptr<FPTC_IDCT_BF16X3, 4>() : nullptr));
    default:
      return nullptr;
  }
}

}  // namespace

uint32_t tc_tile_windows() { return kT; }

// Shared-memory layout of the tensor-core kernel; returns total bytes.
size_t tc_smem_layout(uint32_t mode, uint32_t threads, const uint32_t *lmax, uint32_t n_domains, TcParams *tp) {
  const uint32_t nwg = threads / 128;
  size_t o = 0;
  tp->a_off = 0;
  // one A buffer: 128 x 64 B (TF32), twice that (TF32X3: big, small), or 2 x 128 x 32 B (BF16X3: hi, lo)
  tp->a_buf = mode == FPTC_IDCT_TF32X3 ? 16384u : 8192u;
  tp->a_bytes = 2 * tp->a_buf;         // double buffered
  o += (size_t)nwg * tp->a_bytes;
  tp->b_off = (uint32_t)o;
  o += 4096;                           // up to two 32 x 64-byte operands
  tp->coef_off = (uint32_t)o;
  tp->coef_bytes = (uint32_t)align16((size_t)(kGuard + kTS) * 4 + kGuard + kTS);
  o += (size_t)(threads / 32) * tp->coef_bytes;
  o = align16(o);
  tp->misc_off = (uint32_t)o;
  o += 16 * nwg + 16;
  o = align16(o);
  tp->dom_off = (uint32_t)o;
  o += align16(sizeof(DomTc) * (n_domains ? n_domains : 1));
  tp->tab_first = (uint32_t)o;
  tp->n_domains = n_domains;
  for (uint32_t d = 0; d < n_domains; ++d) o += align16((size_t)2 << lmax[d]) + align16(3u * kZStride * 4);
  return o;
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

cudaError_t launch_tc(const DecodeParams &p, const TcParams &tp, uint32_t mode, uint32_t threads, uint32_t grid,
                      size_t smem, cudaStream_t stream) {
  if (p.tile_end <= p.tile_begin || grid == 0) return cudaSuccess;
  void *k = tcpick(mode, threads);
  if (!k) return cudaErrorInvalidValue;
  DecodeParams pp = p;
  TcParams tt = tp;
  void *args[] = {&pp, &tt};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, stream);
}

}  // namespace fptc
