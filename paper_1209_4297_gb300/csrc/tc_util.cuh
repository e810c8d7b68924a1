// Primitives of the 5th-generation tensor cores (tcgen05), mbarriers and bounded waits,
// shared by the kernels of libridc.so that issue tcgen05.mma from one thread and read their
// FP32 accumulators back from tensor memory. Inline PTX only.
#pragma once

#include <cstdint>

namespace ridc {
namespace tc {

// every device-side wait gives up after this much %globaltimer time and flags the error
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t s_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long s_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool s_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool s_wait(uint32_t bar, uint32_t parity, int* err) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (s_try(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      const unsigned long long t = s_gtimer();
      if (t0 == 0) t0 = t;
      else if (t - t0 > kWaitNs) {
        atomicExch(err, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void s_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// K-major operand tile with 128-byte rows (64 BF16 or 32 FP32 values), 128B swizzle, 8-row
// groups 1 KB apart; the tile starts on a 1 KB boundary
__device__ __forceinline__ uint64_t s_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// kind::f16, BF16 x BF16 -> FP32, both K-major, M = 128, N from the instruction descriptor
__device__ __forceinline__ void s_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void s_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void s_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void s_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void s_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// generic-proxy writes to shared memory become visible to the tensor cores (async proxy)
__device__ __forceinline__ void s_fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// kind::tf32: FP32 operands read as TF32 (both K-major), FP32 accumulator, M = 128
__device__ __forceinline__ void s_mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// tensor-memory allocation of `cols` columns (a power of two >= 32) by one whole warp; the
// base address lands in shared memory at `slot`
__device__ __forceinline__ void s_tmem_alloc(uint32_t slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void s_tmem_free(uint32_t base, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols)
               : "memory");
}

}  // namespace tc
}  // namespace ridc
