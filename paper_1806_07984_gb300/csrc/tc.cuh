// Blackwell tensor-core helpers (tcgen05 MMA with shared-memory operands and
// a TMEM accumulator) for the predictor's derivative contractions.
//
// Operand tiles use the canonical K-major layout without swizzle: a tile of
// R rows x 32 bytes (K = 8 TF32 or K = 16 BF16 values per row) is stored as
// core matrices of 8 rows x 16 bytes (128 contiguous bytes); the two core
// matrices of one 8-row group are adjacent (leading byte offset 128) and
// consecutive 8-row groups are 256 bytes apart (stride byte offset 256).
#pragma once
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ader {
namespace tc {

constexpr uint32_t kLBO = 128;
constexpr uint32_t kSBO = 256;
constexpr int kTileBytes = 128 * 32;  // one M = 128 operand tile

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of (row, kbyte) inside a tile
__host__ __device__ __forceinline__ uint32_t canon(int row, int kbyte) {
  return uint32_t((row >> 3) * kSBO + (kbyte >> 4) * kLBO + (row & 7) * 16 + (kbyte & 15));
}

// shared-memory matrix descriptor (no swizzle, descriptor version 1)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = uint64_t((saddr & 0x3FFFF) >> 4);
  d |= uint64_t((kLBO >> 4) & 0x3FFF) << 16;
  d |= uint64_t((kSBO >> 4) & 0x3FFF) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// instruction descriptor: FP32 accumulator, A/B format fmt (TF32 = 2 for
// kind::tf32, BF16 = 1 for kind::f16), both K-major, shape M x N
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               :: "r"(smem_addr(dst)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int KIND>  // 0: kind::tf32, 1: kind::f16
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, bool acc) {
  if (KIND == 0)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(id), "r"(uint32_t(acc)));
  else
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(id), "r"(uint32_t(acc)));
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_addr(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(mbar)), "r"(count));
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int max_iters) {
  uint32_t done = 0;
  for (int it = 0; it < max_iters; ++it) {
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_addr(mbar)), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// 32 lanes x 8 columns of 32-bit accumulators into 8 registers per thread.
__device__ __forceinline__ void ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Round an FP32 value to TF32 (round to nearest, ties away), kept in FP32 bits.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc
}  // namespace ader
