// fdas_umma.cuh -- tcgen05.mma issue helpers (kind::f16) for the z-band inference kernel.
#pragma once

#include <cstdint>

#include "fdas_device.cuh"

namespace fdas {

// ---------------------------------------------------------------------------------------
// tcgen05.mma (kind::f16, one CTA): D[128 x N] (+)= A[128 x K16] * B[N x K16]^T, operands in
// shared memory in the K-major no-swizzle canonical layout -- core matrices of 8 rows x 16 B
// (rows 16 B apart), core matrices adjacent along K `lbo` bytes apart, 8-row groups along
// M / N `sbo` bytes apart.  The accumulator lives in TMEM.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);   // descriptor version 1, no swizzle
}
// Instruction descriptor: F32 accumulator, F16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive once on `bar` when every tcgen05.mma this thread issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

}  // namespace fdas
