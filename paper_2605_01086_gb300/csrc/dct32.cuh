// The DCT-II of a 32-sample window truncated to 16 bins, as the mirrored
// even/odd split of Eq. 1 (N = 32): with u[n] = x[n] + x[31-n] and
// v[n] = x[n] - x[31-n], the odd bins are sum_n v[n] cos(pi (2n+1) k / 64)
// and the even bins the same construction applied to u (twice more); 232 FP32
// operations with compile-time cosines.  Output a[k] = sum_n x[n] B[k][n] with
// B[0][n] = 1/2 and B[k][n] = cos(pi/N (n + 1/2) k): the adjoint of the
// inverse transform, and Eq. 1 up to the scale 2/N (4/N for bin 0).
// Used by the decoder's adjoint (backward_warp.cu) and the encoder (encode.cu).
//
// Rounding: every intermediate is a signed sum of samples with coefficients of
// magnitude <= 1, so each rounding adds at most 2^-24 sum |x| to the error of
// an output, and an output passes through at most 20 roundings (one
// butterfly level or three, then a chain of at most 16 fused multiply-adds)
// plus its cosines' representation (2^-25 each): |a_fp32[k] - a[k]| <= 2^-19.5
// sum_n |x[n]|.
#pragma once

#include <cmath>
#include <cstdint>

namespace fptc {
namespace dct32 {

// The odd/even cosine groups of the forward transform, read transposed here.
struct AdjK {
  float eee[4];     // cos(pi (2n+1) / 8), n < 4                 (bin 8)
  float eeo[4][2];  // cos(pi (2n+1)(2j+1) / 16)                 (bins 4, 12)
  float eo[8][4];   // cos(pi (2n+1)(2j+1) / 32)                 (bins 2, 6, 10, 14)
  float o[16][8];   // cos(pi (2n+1)(2j+1) / 64)                 (odd bins)
};
__host__ __device__ constexpr double cos_taylor_b(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int i = 1; i < 24; ++i) {
    term *= -x2 / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr float cospi_b(int num, int den) {
  int r = num % (2 * den);
  if (r > den) r = 2 * den - r;
  const double pi = 3.14159265358979323846;
  return 2 * r <= den ? (float)cos_taylor_b(pi * r / den) : (float)-cos_taylor_b(pi * (den - r) / den);
}
__host__ __device__ constexpr AdjK make_adj_k() {
  AdjK K{};
  for (int n = 0; n < 4; ++n) K.eee[n] = cospi_b(2 * n + 1, 8);
  for (int n = 0; n < 4; ++n)
    for (int j = 0; j < 2; ++j) K.eeo[n][j] = cospi_b((2 * n + 1) * (2 * j + 1), 16);
  for (int n = 0; n < 8; ++n)
    for (int j = 0; j < 4; ++j) K.eo[n][j] = cospi_b((2 * n + 1) * (2 * j + 1), 32);
  for (int n = 0; n < 16; ++n)
    for (int j = 0; j < 8; ++j) K.o[n][j] = cospi_b((2 * n + 1) * (2 * j + 1), 64);
  return K;
}

// a[0..15] = gc of one window from its 32 samples (or sample gradients) g.
__device__ __forceinline__ void dct2_16(const float (&g)[32], float (&gc)[16]) {
  constexpr AdjK K = make_adj_k();
  float u[16], v[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    u[n] = g[n] + g[31 - n];
    v[n] = g[n] - g[31 - n];
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {  // odd bins 2j + 1
    float a = v[0] * K.o[0][j];
#pragma unroll
    for (int n = 1; n < 16; ++n) a = fmaf(v[n], K.o[n][j], a);
    gc[2 * j + 1] = a;
  }
  float uu[8], uv[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    uu[n] = u[n] + u[15 - n];
    uv[n] = u[n] - u[15 - n];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {  // bins 4j + 2
    float a = uv[0] * K.eo[0][j];
#pragma unroll
    for (int n = 1; n < 8; ++n) a = fmaf(uv[n], K.eo[n][j], a);
    gc[4 * j + 2] = a;
  }
  float uuu[4], uuv[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    uuu[n] = uu[n] + uu[7 - n];
    uuv[n] = uu[n] - uu[7 - n];
  }
  gc[0] = 0.5f * ((uuu[0] + uuu[1]) + (uuu[2] + uuu[3]));
  {
    float a = uuu[0] * K.eee[0];
#pragma unroll
    for (int n = 1; n < 4; ++n) a = fmaf(uuu[n], K.eee[n], a);
    gc[8] = a;
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {  // bins 4, 12
    float a = uuv[0] * K.eeo[0][j];
#pragma unroll
    for (int n = 1; n < 4; ++n) a = fmaf(uuv[n], K.eeo[n][j], a);
    gc[8 * j + 4] = a;
  }
}


// dct2_16 with a bound on each output's rounding error from the butterfly's
// own intermediate sums (u = 2^-24; K rounded to FP32: |K~ - K| <= 2^-25):
//   odd bins      from v (16-term FMA chains):    18.1 u sum|v|
//   bins 4j + 2   from uv (8-term chains):        u (9.6 sum|uv| + sum|u|)
//   bins 4, 12    from uuv (4-term chains):       u (5.6 sum|uuv| + sum|uu| + sum|u|)
//   bin 8         from uuu (4-term chain):        u (5.6 sum|uuu| + sum|uu| + sum|u|)
//   bin 0         1/2 of three sums of uuu:       u (1.5 sum|uuu| + sum|uu| + sum|u|) / 2 + ...
// Each intermediate w = fl(p +- q) carries |w~ - w| <= u |w| plus the errors
// of p and q; a chain of m fused multiply-adds adds at most 1.01 m u sum |input|
// and the cosines' rounding 0.5 u sum |input|.  For signals with an offset the
// DC cancels in v and uv, so these are much tighter than a multiple of
// sum |x|.  e[k] bounds |a_fp32[k] - a[k]| with 2 % to spare (the sums are
// themselves rounded).
__device__ __forceinline__ void dct2_16_bounded(const float (&g)[32], float (&gc)[16], float (&e)[16]) {
  constexpr AdjK K = make_adj_k();
  constexpr float u = 0x1p-24f * 1.02f;
  float uu_[16], v[16];
  float su = 0.0f, sv = 0.0f;
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    uu_[n] = g[n] + g[31 - n];
    v[n] = g[n] - g[31 - n];
    su += fabsf(uu_[n]);
    sv += fabsf(v[n]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {  // odd bins 2j + 1
    float a = v[0] * K.o[0][j];
#pragma unroll
    for (int n = 1; n < 16; ++n) a = fmaf(v[n], K.o[n][j], a);
    gc[2 * j + 1] = a;
    e[2 * j + 1] = 18.1f * u * sv;
  }
  float uu[8], uv[8];
  float suu = 0.0f, suv = 0.0f;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    uu[n] = uu_[n] + uu_[15 - n];
    uv[n] = uu_[n] - uu_[15 - n];
    suu += fabsf(uu[n]);
    suv += fabsf(uv[n]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {  // bins 4j + 2
    float a = uv[0] * K.eo[0][j];
#pragma unroll
    for (int n = 1; n < 8; ++n) a = fmaf(uv[n], K.eo[n][j], a);
    gc[4 * j + 2] = a;
    e[4 * j + 2] = u * (9.6f * suv + su);
  }
  float uuu[4], uuv[4];
  float suuu = 0.0f, suuv = 0.0f;
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    uuu[n] = uu[n] + uu[7 - n];
    uuv[n] = uu[n] - uu[7 - n];
    suuu += fabsf(uuu[n]);
    suuv += fabsf(uuv[n]);
  }
  gc[0] = 0.5f * ((uuu[0] + uuu[1]) + (uuu[2] + uuu[3]));
  e[0] = 0.5f * u * (3.0f * suuu + suu + su);
  {
    float a = uuu[0] * K.eee[0];
#pragma unroll
    for (int n = 1; n < 4; ++n) a = fmaf(uuu[n], K.eee[n], a);
    gc[8] = a;
    e[8] = u * (5.6f * suuu + suu + su);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {  // bins 4, 12
    float a = uuv[0] * K.eeo[0][j];
#pragma unroll
    for (int n = 1; n < 4; ++n) a = fmaf(uuv[n], K.eeo[n][j], a);
    gc[8 * j + 4] = a;
    e[8 * j + 4] = u * (5.6f * suuv + suu + su);
  }
}

}  // namespace dct32
}  // namespace fptc
