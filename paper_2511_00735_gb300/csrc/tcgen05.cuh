// Device helpers shared by the tcgen05 kernels (tc.cu, ozk.cu): shared-memory addresses,
// bounded mbarrier waits, asynchronous and bulk copies, the 16-bit K-major no-swizzle tile
// layout and its descriptor, and the kind::f16 MMA.
#pragma once

#include <cstdint>

namespace hps {
namespace tcg {

// iterations of an mbarrier try_wait loop before a wait gives up
constexpr long long WAIT_LIMIT = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// true once the phase of the given parity has completed; false after WAIT_LIMIT tries
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < WAIT_LIMIT && !done; ++it)
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done)
                 : "r"(mbar), "r"(parity)
                 : "memory");
  return done != 0;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_u32(b)) : "memory");
}
// one arrival on b that also expects `bytes` of bulk copies to complete on it
__device__ __forceinline__ void expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16) completing on b
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}
// arrive on b once every tcgen05 operation this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// arrive on b once every cp.async this thread issued so far has landed (the arrival is counted in
// the barrier's initial count)
__device__ __forceinline__ void cp_async_arrive(uint64_t* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
// 8-byte asynchronous copy that reads nbytes (0 or 8) from src and zero-fills the rest, so that
// padding reaches shared memory through the same completion mechanism as the data
__device__ __forceinline__ void cp_async8z(uint32_t dst, const void* src, uint32_t nbytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(nbytes) : "memory");
}
// the same with 16 bytes (16-byte aligned addresses; nbytes 0, 8 or 16)
__device__ __forceinline__ void cp_async16z(uint32_t dst, const void* src, uint32_t nbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(nbytes) : "memory");
}

// 16-bit K-major no-swizzle tiles: 8-row x 16-byte core matrices, LBO16 bytes apart along k and
// SBO16 apart between 8-row groups (16 elements of k = two core matrices per row group)
constexpr uint32_t LBO16 = 128;
constexpr uint32_t SBO16 = 256;

// byte offset of the 16-bit element (r, k) of a tile
__device__ __forceinline__ uint32_t core_off16(int r, int k) {
  return (uint32_t)(r >> 3) * SBO16 + (uint32_t)(k >> 3) * LBO16 + (uint32_t)(r & 7) * 16 + (uint32_t)(k & 7) * 2;
}
// shared-memory matrix descriptor of such a tile: start >> 4, LBO >> 4, SBO >> 4, version 1
__device__ __forceinline__ uint64_t smem_desc16(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(LBO16 >> 4) << 16) | ((uint64_t)(SBO16 >> 4) << 32) |
         ((uint64_t)1 << 46);
}
// D (tensor memory, FP32) (+)= A * B, kind::f16 (A, B from shared-memory descriptors)
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate) {
  asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                   tmem),
               "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
               : "memory");
}

}  // namespace tcg
}  // namespace hps
