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
// seven G_s are combined exactly in 128-bit integers and rounded once to FP64.
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
constexpr uint32_t BAR_OFF = E_OFF + 192 * 4;
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

// The seven signed digits of x relative to 2^e (digit 0 most significant).
__device__ __forceinline__ void digits(double x, int e, int (&n)[S]) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long X = 0;
  if (E != 0 && e != ZERO_ROW) {
    const unsigned long long M = (unsigned long long)(b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 4 + (E - 1023) - e;  // X = floor(|x| 2^{56 - e}) = M 2^sh, sh <= 3
    X = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> (-sh)) : 0ull);
  }
  int carry = 0;
#pragma unroll
  for (int i = S - 1; i >= 0; --i) {
    int v = (int)((X >> (8 * (S - 1 - i))) & 0xFFull) + carry;
    carry = 0;
    if (i > 0 && v >= 128) {
      v -= 256;
      carry = 1;
    }
    n[i] = v;
  }
  if (b < 0) {
#pragma unroll
    for (int i = 0; i < S; ++i) n[i] = -n[i];
  }
}

// Rows [row0, row0 + 64) of the operand from a row-major 64 x 64 FP64 tile
// `src`: thread t < 64 of the calling group handles row t.  Writes the seven
// digit slices (bf16) and the row exponent.
__device__ __forceinline__ void stage_row(unsigned char* slices, uint32_t slice_bytes, int* ex,
                                          const double* __restrict__ src, int r, int row) {
  const double2* p = reinterpret_cast<const double2*>(src + r * 64);
  double m = 0.0;
#pragma unroll 8
  for (int q = 0; q < 32; ++q) {
    const double2 v = p[q];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  const int e = row_exponent(m);
  ex[row] = e;
  for (int c8 = 0; c8 < 8; ++c8) {
    uint32_t w[S][4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const double2 v = p[4 * c8 + h];
      int n0[S], n1[S];
      digits(v.x, e, n0);
      digits(v.y, e, n1);
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const uint32_t lo = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)n0[i]));
        const uint32_t hi = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)n1[i]));
        w[i][h] = lo | (hi << 16);
      }
    }
    const uint32_t off = core_offset(row, c8);
#pragma unroll
    for (int i = 0; i < S; ++i)
      *reinterpret_cast<uint4*>(slices + (size_t)i * slice_bytes + off) =
          make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
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

// 2^{er + ec} (hi 2^{-40} + lo 2^{-64}) rounded once to FP64, with
// hi = sum_{s<=3} G_s 2^{8(3-s)}, lo = sum_{s>=4} G_s 2^{8(6-s)}.
__device__ __forceinline__ double combine(long long hi, long long lo, int er, int ec) {
  const __int128 V = (__int128)hi * ((__int128)1 << 24) + (__int128)lo;  // value = V 2^{er + ec - 64}
  if (V == 0) return 0.0;
  const bool neg = V < 0;
  const unsigned __int128 U = neg ? (unsigned __int128)(-V) : (unsigned __int128)V;
  const unsigned long long uh = (unsigned long long)(U >> 64), ul = (unsigned long long)U;
  const int msb = uh ? 127 - __clzll((long long)uh) : 63 - __clzll((long long)ul);
  unsigned long long m;
  int top = msb;
  if (msb <= 52) {
    m = ul << (52 - msb);
  } else {
    const int sh = msb - 52;
    m = (unsigned long long)(U >> sh);
    const unsigned __int128 rem = U & (((unsigned __int128)1 << sh) - 1);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m == (1ull << 53)) {
      m >>= 1;
      ++top;
    }
  }
  const int E = top + er + ec - 64 + 1023;
  if (E <= 0 || E >= 2047) {  // outside the normal range: scale in FP64
    const double mant = (double)(long long)m * (neg ? -1.0 : 1.0);
    return ldexp(mant, top - 52 + er + ec - 64);
  }
  const unsigned long long bits =
      (neg ? (1ull << 63) : 0ull) | ((unsigned long long)E << 52) | (m & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// 16 accumulator columns [c0, c0 + 16) of this thread's lane for every group,
// combined into FP64 values v[16] (column scales ec[c0 + j]).
__device__ __forceinline__ void read_combine16(uint32_t tmem_lane, int c0, int er,
                                               const int* ecols, double (&v)[16]) {
  long long hi[16], lo[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0;
#pragma unroll
  for (int s = 0; s < NG; ++s) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(tmem_lane + 64u * s + (uint32_t)c0)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const long long g = (long long)__float2int_rn(__uint_as_float(r[j]));
      if (s <= 3) hi[j] += g * (1ll << (8 * (3 - s)));
      else lo[j] += g * (1ll << (8 * (6 - s)));
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j)
    v[j] = (er == ZERO_ROW || ecols[c0 + j] == ZERO_ROW) ? 0.0
                                                         : combine(hi[j], lo[j], er, ecols[c0 + j]);
}

}  // namespace oz
}  // namespace sfcdd
