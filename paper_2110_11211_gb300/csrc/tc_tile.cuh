// Tile products on the 5th-generation tensor cores (tcgen05) for the FP32
// local factorization: D (128 x 64, FP32, in tensor memory) = A B^T with
// A = two stacked 64 x 64 row-major tiles and B one 64 x 64 tile, K = 64.
//
// FP32 accuracy from TF32 operands by the error-compensated split (x ~= hi + lo,
// hi = x rounded to TF32, lo = x - hi rounded to TF32, so |x - hi - lo| <=
// 2^-22 |x|):
//   A B^T ~= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// (the dropped A_lo B_lo^T term is 2^-22 relative to |A||B^T|), accumulated in
// FP32 in tensor memory.
//
// Shared-memory operand layout: K-major without swizzle, in core matrices of
// 8 rows x 16 bytes (8 x 4 FP32).  Row r, column c of an operand sits at byte
//   (r / 8) * SBO + (c / 4) * LBO + (r % 8) * 16 + (c % 4) * 4,
// LBO = 128 (core matrices adjacent along K), SBO = 16 * 128 = 2048 (row groups),
// so a 64 x 64 tile takes 16 KB and a 128 x 64 operand 32 KB.  One MMA consumes
// K = 8 (two core matrices along K); step s starts s * 256 bytes further.
//
// Accumulator layout (M = 128, one CTA): row i of D in tensor-memory lane i,
// column j in column j.  Warp w reads lanes 32 (w % 4) .. + 31.
#pragma once

#include <cstdint>

namespace sfcdd {
namespace tc {

constexpr int TC_M = 128;
constexpr int TC_N = 64;
constexpr int TC_K = 64;
constexpr uint32_t LBO = 128;
constexpr uint32_t SBO = 2048;
constexpr uint32_t A_BYTES = TC_M * TC_K * 4;  // 32 KB
constexpr uint32_t B_BYTES = TC_N * TC_K * 4;  // 16 KB
// A_hi | A_lo | B_hi | B_lo, then the mbarrier and the tensor-memory address
constexpr uint32_t SMEM_BYTES = 2 * A_BYTES + 2 * B_BYTES + 16;
constexpr uint32_t TMEM_COLS = 64;

// Instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), LBO >> 4
// (bits 16-29), SBO >> 4 (bits 32-45), descriptor version 1 (bit 46), no
// swizzle (bits 61-63 = 0), base offset 0.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((LBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t core_offset(int r, int c) {
  return (uint32_t)((r >> 3) * SBO + (c >> 2) * LBO + (r & 7) * 16 + (c & 3) * 4);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}

// Stage 64 rows of a row-major 64 x 64 FP32 tile as rows [row0, row0 + 64) of
// an operand, split into hi and lo.  All threads of the CTA take part.
__device__ __forceinline__ void stage_tile(unsigned char* hi, unsigned char* lo,
                                           const float* __restrict__ src, int row0) {
  for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
    const int r = e >> 4, c4 = (e & 15) * 4;
    const float4 v = *reinterpret_cast<const float4*>(src + r * 64 + c4);
    float4 h, l;
    h.x = tf32_round(v.x);
    h.y = tf32_round(v.y);
    h.z = tf32_round(v.z);
    h.w = tf32_round(v.w);
    l.x = tf32_round(v.x - h.x);
    l.y = tf32_round(v.y - h.y);
    l.z = tf32_round(v.z - h.z);
    l.w = tf32_round(v.w - h.w);
    const uint32_t off = core_offset(row0 + r, c4);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait on phase `ph` of an mbarrier; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t ph, long long limit) {
  const uint32_t a = smem_addr(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(ph)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(128);
  }
  return false;
}

// Whole warp: allocate TMEM_COLS columns, address written to *dst (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(dst)),
               "r"(TMEM_COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
               "r"(TMEM_COLS)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes made visible to the tensor core's reads.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

// Issue the 3 x 8 MMAs of D = A B^T (error-compensated split); one thread.
__device__ __forceinline__ void issue_product(uint32_t tmem_d, const unsigned char* ahi,
                                              const unsigned char* alo, const unsigned char* bhi,
                                              const unsigned char* blo) {
  const uint32_t a0 = smem_addr(ahi), a1 = smem_addr(alo), b0 = smem_addr(bhi),
                 b1 = smem_addr(blo);
#pragma unroll
  for (int s = 0; s < TC_K / 8; ++s) {
    const uint32_t o = (uint32_t)s * 2 * LBO;
    mma_tf32(tmem_d, make_desc(a1 + o), make_desc(b0 + o), s > 0);  // A_lo B_hi
    mma_tf32(tmem_d, make_desc(a0 + o), make_desc(b1 + o), 1);      // A_hi B_lo
    mma_tf32(tmem_d, make_desc(a0 + o), make_desc(b0 + o), 1);      // A_hi B_hi
  }
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace sfcdd
