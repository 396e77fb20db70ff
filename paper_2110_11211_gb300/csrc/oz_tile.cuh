// FP64 tile products D = A B^T on the bf16 tensor cores by exact slicing
// (the error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", 2012), for the FP64 factorizations.
//
// Each row x of A (and of B) is scaled by its own power of two 2^e, e = the
// exponent with max|x| < 2^e, and its entries are cut into S = 7 signed 8-bit
// digits:  x_k = 2^e sum_{i<7} n_{k,i} 2^{-8(i+1)} + t_k,  |t_k| < 2^{e-56},
// n_{k,0} in [-256, 256], n_{k,i>0} in [-128, 127] (a signed-digit recoding of
// the 56-bit truncated magnitude, done with integer operations on the bit
// pattern).  Every digit is exact in bf16.  Then
//   (A B^T)_{rc} ~= 2^{e_r + e_c} sum_{s=0}^{6} 2^{-8(s+2)} G_s[r][c],
//   G_s = sum_{i+j=s} sum_k n^A_{r,k,i} n^B_{c,k,j},
// each G_s formed by bf16 MMAs with FP32 accumulation in tensor memory.  The
// products are integers bounded by 2^16 (2^15 off the leading digits), so
// |G_s| <= 64 (2^16 + 5 2^14) < 2^24 and every accumulation is exact.  The
// dropped terms (digit pairs with i + j > 6 and the truncation t) are below
// 2^-55 |A| |B^T| relative, the size of one FP64 rounding of the sum.  The
// seven G_s are combined in one 64-bit integer and rounded once to FP64.
//
// Shared-memory operand layout (bf16, K-major, no swizzle): core matrices of
// 8 rows x 16 bytes (8 x 8 bf16); row r, column c of a slice at byte
//   (r / 8) * 1024 + (c / 8) * 128 + (r % 8) * 16 + (c % 8) * 2,
// LBO = 128, SBO = 1024: 16 KB per 128-row slice, 8 KB per 64-row slice.  One
// MMA consumes K = 16.  Accumulator of group s: tensor-memory columns
// [64 s, 64 s + 64), row i of D in lane i (M = 128).
#pragma once

#include <cstdint>

#include "tc_tile.cuh"

namespace sfcdd {
namespace oz {

constexpr int S = 7;                     // digits per entry
constexpr int NG = S;                    // digit-pair groups s = i + j <= S - 1
constexpr uint32_t LBO = 128;
constexpr uint32_t SBO = 1024;
constexpr uint32_t A_SLICE = 128 * 64 * 2;  // 16 KB
constexpr uint32_t B_SLICE = 64 * 64 * 2;   // 8 KB
constexpr uint32_t A_OFF = 0;
constexpr uint32_t B_OFF = S * A_SLICE;                 // 112 KB
constexpr uint32_t E_OFF = B_OFF + S * B_SLICE;         // 168 KB: row exponents (192 ints)
constexpr uint32_t MAX_OFF = E_OFF + 192 * 4;           // row maxima as bit patterns (192 u64)
constexpr uint32_t BAR_OFF = MAX_OFF + 192 * 8;
constexpr uint32_t SMEM_BYTES = BAR_OFF + 16;
constexpr uint32_t TMEM_COLS = 512;  // 7 groups x 64 columns, rounded up
constexpr int ZERO_ROW = -100000;    // exponent of an all-zero row

// kind::f16 with bf16 A and B (bits 7-9, 10-12 = 1), FP32 D, K-major, N = 64, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (8u << 17) | (8u << 24);

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((LBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t core_offset(int r, int c8) {
  return (uint32_t)((r >> 3) * SBO + c8 * LBO + (r & 7) * 16);
}

// e with max|x| < 2^e (ZERO_ROW for an all-zero row); subnormal maxima count as zero.
__device__ __forceinline__ int row_exponent(double maxabs) {
  const long long b = __double_as_longlong(maxabs);
  const int E = (int)((b >> 52) & 0x7FF);
  return E == 0 ? ZERO_ROW : E - 1022;
}

// bf16 bit pattern of an integer n with |n| <= 256 (exact): 0x4B400000 + n is
// the FP32 pattern of 1.5 2^23 + n, so subtracting 1.5 2^23 in FP32 gives n
// exactly; n has at most 9 significant bits, so its FP32 pattern ends in 16 zeros.
__device__ __forceinline__ uint32_t bf16_of_int(int n) {
  const float f = __int_as_float(0x4B400000 + n) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

// The seven balanced digits of x relative to 2^e, as bf16 bit patterns: with
// X = floor(|x| 2^{56 - e}) and Y = X + 0x808080808080 (128 added to the six low
// bytes), digit 0 is Y >> 48 in [0, 256] and digit i > 0 is byte 6 - i of Y minus
// 128, in [-128, 127]; sum_i digit_i 2^{8(6-i)} = X exactly; the sign of x is
// applied to every digit.
__device__ __forceinline__ void digits_bf16(double x, int e, uint32_t (&d)[S]) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long X = 0;
  if (E != 0 && e != ZERO_ROW) {
    const unsigned long long M = (unsigned long long)(b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 4 + (E - 1023) - e;
    X = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> (-sh)) : 0ull);
  }
  const unsigned long long Y = X + 0x808080808080ull;
  const uint32_t yh = (uint32_t)(Y >> 32), yl = (uint32_t)Y;
  const int sg = b < 0 ? -1 : 1;
  d[0] = bf16_of_int(sg * (int)(yh >> 16));
  d[1] = bf16_of_int(sg * ((int)((yh >> 8) & 0xFFu) - 128));
  d[2] = bf16_of_int(sg * ((int)(yh & 0xFFu) - 128));
  d[3] = bf16_of_int(sg * ((int)(yl >> 24) - 128));
  d[4] = bf16_of_int(sg * ((int)((yl >> 16) & 0xFFu) - 128));
  d[5] = bf16_of_int(sg * ((int)((yl >> 8) & 0xFFu) - 128));
  d[6] = bf16_of_int(sg * ((int)(yl & 0xFFu) - 128));
}

// Stage the 192 operand rows (A: rows 0-63 of a0, rows 64-127 of a1; B: rows of b)
// as digit slices, every thread of the CTA taking six (row, 8-column chunk)
// tasks: a warp covers 8 rows x 4 chunks, so its loads are 256-byte row pieces
// and its 16-byte slice stores fill whole 128-byte lines.  All loads are issued
// first and kept in registers; the row maxima come from shared atomics on the
// bit patterns of |x| (which order like the values), then the digits are written.
__device__ __forceinline__ void stage_all(unsigned char* dsm, const double* __restrict__ a0,
                                          const double* __restrict__ a1,
                                          const double* __restrict__ b) {
  int* ex = reinterpret_cast<int*>(dsm + E_OFF);
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(dsm + MAX_OFF);
  for (int i = threadIdx.x; i < 192; i += blockDim.x) mx[i] = 0ull;
  __syncthreads();
  constexpr int NT = 192 * 8;
  constexpr int PER = NT / 256;  // tasks per thread (the kernels run 256 threads)
  ulonglong2 v[PER][4];
  int rows[PER], cs[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int T = threadIdx.x + 256 * j;
    const int g = T >> 6, w = T & 63;
    const int row = 8 * g + (w & 7), c = 4 * (w >> 5) + ((w & 31) >> 3);
    rows[j] = row;
    cs[j] = c;
    const double* src = row < 64 ? a0 + row * 64 : row < 128 ? a1 + (row - 64) * 64 : b + (row - 128) * 64;
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(src + 8 * c);
#pragma unroll
    for (int h = 0; h < 4; ++h) v[j][h] = p[h];
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    unsigned long long m = 0ull;
#pragma unroll
    for (int h = 0; h < 4; ++h)
      m = max(m, max(v[j][h].x & 0x7FFFFFFFFFFFFFFFull, v[j][h].y & 0x7FFFFFFFFFFFFFFFull));
    atomicMax(&mx[rows[j]], m);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 192; i += blockDim.x)
    ex[i] = row_exponent(__longlong_as_double((long long)mx[i]));
  __syncthreads();
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int row = rows[j];
    const int e = ex[row];
    uint32_t wd[S][4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      uint32_t d0[S], d1[S];
      digits_bf16(__longlong_as_double((long long)v[j][h].x), e, d0);
      digits_bf16(__longlong_as_double((long long)v[j][h].y), e, d1);
#pragma unroll
      for (int i = 0; i < S; ++i) wd[i][h] = d0[i] | (d1[i] << 16);
    }
    unsigned char* base = row < 128 ? dsm + A_OFF : dsm + B_OFF;
    const uint32_t sl = row < 128 ? A_SLICE : B_SLICE;
    const uint32_t off = core_offset(row < 128 ? row : row - 128, cs[j]);
#pragma unroll
    for (int i = 0; i < S; ++i)
      *reinterpret_cast<uint4*>(base + (size_t)i * sl + off) =
          make_uint4(wd[i][0], wd[i][1], wd[i][2], wd[i][3]);
  }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

// The 28 digit-pair products of D = A B^T, four K steps each, grouped by s = i + j.
__device__ __forceinline__ void issue_products(uint32_t tmem, uint32_t abase, uint32_t bbase) {
  for (int s = 0; s < NG; ++s) {
    bool first = true;
    for (int i = 0; i <= s; ++i) {
      const int j = s - i;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = (uint32_t)kk * 2 * LBO;
        mma_bf16(tmem + 64u * s, make_desc(abase + i * A_SLICE + o),
                 make_desc(bbase + j * B_SLICE + o), first ? 0u : 1u);
        first = false;
      }
    }
  }
}

// An exact integer |g| < 2^24 held as FP32 bits (a group sum), read with integer
// instructions.
__device__ __forceinline__ long long int_of_f32(uint32_t b) {
  if ((b & 0x7FFFFFFFu) == 0u) return 0;
  const int e = (int)((b >> 23) & 0xFFu) - 127;  // 0..23
  const long long mag = (long long)(((b & 0x7FFFFFu) | 0x800000u) >> (23 - e));
  return (b >> 31) ? -mag : mag;
}

// 8 accumulator columns [c0, c0 + 8) of this thread's lane for every group (the
// seven loads issued back to back, one wait), combined into FP64 values v[8]:
//   D = 2^{er + ec} sum_s 2^{-8(s+2)} G_s = W 2^{er + ec - 54},
//   W = sum_s G_s 2^{8(6-s) - 10}   (|W| < 2^61),
// where the two lowest groups are shifted right (dropping bits below 2^-74 of
// 2^{er + ec}, far below an FP64 rounding of D); W is converted once, to nearest,
// and scaled by adding to the exponent field.
__device__ __forceinline__ void read_combine8(uint32_t tmem_lane, int c0, int er,
                                              const int* ecols, double (&v)[8]) {
  uint32_t r[NG][8];
#pragma unroll
  for (int s = 0; s < NG; ++s)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[s][0]), "=r"(r[s][1]), "=r"(r[s][2]), "=r"(r[s][3]), "=r"(r[s][4]),
          "=r"(r[s][5]), "=r"(r[s][6]), "=r"(r[s][7])
        : "r"(tmem_lane + 64u * s + (uint32_t)c0)
        : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    long long W = 0;
#pragma unroll
    for (int s = 0; s < NG; ++s) {
      const long long g = int_of_f32(r[s][j]);
      const int sh = 8 * (6 - s) - 10;  // 38, 30, 22, 14, 6, -2, -10
      W += sh >= 0 ? g * (1ll << sh) : (g >> (-sh));
    }
    const int ec = ecols[c0 + j];
    double d = 0.0;
    if (W != 0 && er != ZERO_ROW && ec != ZERO_ROW) {
      d = __ll2double_rn(W);
      const int E = (int)((__double_as_longlong(d) >> 52) & 0x7FF) + er + ec - 54;
      d = (E > 0 && E < 2047)
              ? __longlong_as_double(__double_as_longlong(d) + ((long long)(er + ec - 54) << 52))
              : ldexp(d, er + ec - 54);
    }
    v[j] = d;
  }
}

}  // namespace oz
}  // namespace sfcdd
