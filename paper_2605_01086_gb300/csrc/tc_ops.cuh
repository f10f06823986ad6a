// tcgen05 building blocks shared by the tensor-core decode kernels
// (decode_tc.cu, decode_tcs.cu): barriers, fences, shared-memory and instruction
// descriptors, the MMA / tensor-memory load and store wrappers, the operand
// split of each precision form, the products of one 128-window step, and the B
// operand (the inverse-transform basis) in shared memory.
//
// The inverse transform of Eq. 1 for N = 32, E = 16 is
//      D[128 windows x 32 samples] = C[128 x 16 bins] * B[16 x 32],
// B[k][n] = cos(pi/N (n + 1/2) k) (B[0][n] = 1/2).  Precision forms (FP32
// accumulate in every one):
//   TF32    one product, operands rounded to TF32 (10-bit mantissa);
//   TF32X3  C = C_big + C_small, B = B_big + B_small (TF32 each), three
//           products C_big B_big + C_big B_small + C_small B_big;
//   BF16X3  the same split with BF16 halves, C_hi B_hi + C_lo B_hi + C_hi B_lo.
// A lives in tensor memory (one row per lane), B in shared memory, K-major, no
// swizzle: a core matrix is 8 rows x 16 bytes stored contiguously; LBO = byte
// distance between core matrices adjacent in K, SBO = between core matrices
// adjacent in N.
#pragma once

#include <cuda_bf16.h>

#include "warp_tile.cuh"

namespace fptc {
namespace tcx {

using namespace wt;

constexpr int kRows = 128;  // windows per product (MMA M)

// ---- small PTX wrappers -----------------------------------------------------

// Barrier over the 128 threads of named barrier ID returning the OR of v.  The
// id is a compile-time constant: a run-time id makes the compiler reserve every
// hardware barrier of the SM for one CTA.
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

// Barrier over the 128 threads of warpgroup wg (ids 1..7), returning the OR of v.
__device__ __forceinline__ bool wg_barrier_any(uint32_t wg, bool v) {
  switch (wg) {
    case 0: return bar_any_c<1>(v);
    case 1: return bar_any_c<2>(v);
    case 2: return bar_any_c<3>(v);
    case 3: return bar_any_c<4>(v);
    case 4: return bar_any_c<5>(v);
    case 5: return bar_any_c<6>(v);
    default: return bar_any_c<7>(v);
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

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

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Thread i of the warp writes 8 or 16 consecutive 32-bit columns of lane
// (taddr lane) + i.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

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

// Thread i of the warp reads 16 consecutive 32-bit columns of lane (taddr lane) + i.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// ---- operand layouts ---------------------------------------------------------
// B in shared memory.  TF32 (4 bytes): row n, bin k -> (n/8)*512 + (k/4)*128 + (n%8)*16 + (k%4)*4;
// LBO 128, SBO 512.  BF16 (2 bytes): row n, bin k -> (n/8)*256 + (k/8)*128 + (n%8)*16 + (k%8)*2;
// LBO 128, SBO 256.
// A in tensor memory: columns per A set (one step's operands).
template <int MODE>
__host__ __device__ constexpr uint32_t a_cols() {
  return MODE == FPTC_IDCT_TF32X3 ? 32u : 16u;  // BF16X3: hi 8 + lo 8; TF32: 16; TF32X3: big 16 + small 16
}
// Tensor-memory columns per warpgroup: one 32-column D and two A sets.
template <int MODE>
__host__ __device__ constexpr uint32_t wg_cols() {
  return 32u + 2u * a_cols<MODE>();
}

// This lane's row of the A operand(s) from one window's 16 coefficients; a
// points at lane 32 q + i of the A set (all 32 lanes of the warp take part).
template <int MODE>
__device__ __forceinline__ void put_a_row(uint32_t a, const float (&c)[16]) {
  if (MODE == FPTC_IDCT_BF16X3) {
    uint32_t h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float x0 = c[2 * j], x1 = c[2 * j + 1];
      h[j] = pack_bf16(x0, x1);
      const float h0 = __uint_as_float(h[j] << 16), h1 = __uint_as_float(h[j] & 0xffff0000u);
      l[j] = pack_bf16(x0 - h0, x1 - h1);
    }
    tmem_st8(a, h);
    tmem_st8(a + 8, l);
  } else if (MODE == FPTC_IDCT_TF32X3) {
    // big = c with its 13 low mantissa bits cleared (a TF32 value), small = c - big
    // exactly (at most 13 significant bits); the product reads small as TF32, which
    // keeps its top 11 significant bits: |error| <= 2^-10 |small| <= 2^-20 |c|
    uint32_t big[16], sm[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      big[j] = __float_as_uint(c[j]) & 0xFFFFE000u;
      sm[j] = __float_as_uint(c[j] - __uint_as_float(big[j]));
    }
    tmem_st16(a, big);
    tmem_st16(a + 16, sm);
  } else {
    uint32_t big[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) big[j] = __float_as_uint(tf32_round(c[j]));
    tmem_st16(a, big);
  }
}

// The products of one step: A set at tensor-memory column a, B at b, accumulator d.
template <int MODE>
__device__ __forceinline__ void issue_products(uint32_t a, uint32_t b, uint32_t d) {
  if (MODE == FPTC_IDCT_BF16X3) {
    constexpr uint32_t id = instr_desc(kFmtBF16, kRows, kN);
    mma_f16(d, a, smem_desc(b, 128, 256), id, 0);            // hi * hi
    mma_f16(d, a + 8, smem_desc(b, 128, 256), id, 1);        // lo * hi
    mma_f16(d, a, smem_desc(b + 1024, 128, 256), id, 1);     // hi * lo
  } else {
    constexpr uint32_t id = instr_desc(kFmtTF32, kRows, kN);
#pragma unroll
    for (uint32_t h = 0; h < 2; ++h) {  // bins 0..7, 8..15
      mma_tf32(d, a + 8 * h, smem_desc(b + 256 * h, 128, 512), id, h);
      if (MODE == FPTC_IDCT_TF32X3) {
        mma_tf32(d, a + 8 * h, smem_desc(b + 2048 + 256 * h, 128, 512), id, 1);
        mma_tf32(d, a + 16 + 8 * h, smem_desc(b + 256 * h, 128, 512), id, 1);
      }
    }
  }
}

// Output bookkeeping of a step whose product is in flight: where its 32
// windows go (nothing when nwin == 0).
struct StepOut {
  uint64_t out_row;   // output offset of window 0 of the step, in 32-float rows (valid for TMA)
  float *dst;         // first sample of window 0 of the step
  uint64_t left;      // samples of the segment from window 0 of the step on
  uint32_t nwin;      // windows of the step (0..32)
  uint32_t flags;     // bit 0: 16-byte stores, bit 1: 32-byte stores, bit 2: TMA
};

// The B operand(s) of form MODE in shared memory at b_base from the FP32 basis
// [k][n] (k < 16, n < 32), by threads tid = t0, t0 + stride, ...
template <int MODE>
__device__ __forceinline__ void fill_b_operand(unsigned char *b_base, const float *bsrc, uint32_t t0,
                                               uint32_t stride) {
  for (uint32_t i = t0; i < kN * kE; i += stride) {
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

}  // namespace tcx
}  // namespace fptc
