// tcgen05.cuh -- shared pieces of the tensor-core kernels (sm_103a): operand layout,
// shared-memory and instruction descriptors of tcgen05.mma kind::f16, the BF16 hi/lo split
// and bounded mbarrier waits.  Inline PTX only.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace afmpb {

constexpr uint32_t kTcSpinLimit = 1u << 26;    // polls of a bounded mbarrier wait

// Byte offset of element (row, k) in a canonical K-major no-swizzle tile with `rows` rows.
__host__ __device__ __forceinline__ uint32_t canon_off(int row, int k, int rows) {
  return (uint32_t)((((k >> 3) * (rows >> 3) + (row >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;                       // descriptor version for tcgen05
  return d;                                     // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  uint32_t d = 0;
  d |= 1u << 4;                                 // D format F32
  d |= 1u << 7;                                 // A format BF16
  d |= 1u << 10;                                // B format BF16
  d |= (uint32_t)(N >> 3) << 17;
  d |= (uint32_t)(M >> 4) << 24;
  return d;
}

__device__ __forceinline__ uint32_t cvta_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, uint32_t limit = kTcSpinLimit) {
  for (uint32_t spin = 0; spin < limit; ++spin) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(mb), "r"(parity));
    if (ok) return true;
  }
  return false;
}

// 16-byte global -> shared copy; valid == false fills the 16 bytes with zeros instead
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

}  // namespace afmpb
