// Helpers for the 5th-generation tensor cores (tcgen05) shared by the
// dense block (dense.cu) and the ensemble density matrix (rho_tc.cu):
// bf16 operands in shared memory in the canonical K-major layout without
// swizzle, one 128 x 64 FP32 accumulator per 64 tensor-memory columns.
//
// Canonical layout of a tile of R rows x 64 bf16 (one K chunk): 8-row x
// 16-byte core matrices (8 bf16 along K), 128 contiguous bytes each; core
// matrices adjacent in K are 128 B apart (leading byte offset), 8-row groups
// 8 x 128 = 1024 B apart (stride byte offset).  One MMA takes K = 16 (two
// core matrices along K), M = 128 rows of A and N = 64 rows of B.
#pragma once

#include <stdint.h>

namespace qc {

#define TC5_M 128
#define TC5_N 64
#define TC5_K 64
#define TC5_LBO 128
#define TC5_SBO 1024
#define TC5_A_SLICE (TC5_M * TC5_K * 2)  // 16 KiB: one digit slice of a 128-row tile
#define TC5_B_SLICE (TC5_N * TC5_K * 2)  // 8 KiB: one digit slice of a 64-row tile

__host__ __device__ __forceinline__ uint32_t tc5_canon_off(int r, int k) {  // byte offset of bf16 (row r, column k)
  return (uint32_t)((r >> 3) * TC5_SBO + (k >> 3) * TC5_LBO + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t tc5_smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(TC5_LBO >> 4) << 16) |
         ((uint64_t)(TC5_SBO >> 4) << 32) | (1ull << 46);  // descriptor version 1, no swizzle (layout 0)
}

// kind::f16, D = F32, A = B = BF16, both K-major, N = 64, M = 128
#define TC5_IDESC ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC5_N >> 3) << 17) | ((uint32_t)(TC5_M >> 4) << 24))

__device__ __forceinline__ void tc5_mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(TC5_IDESC), "r"(acc));
}

// Polls an mbarrier phase at most `limit` times; false if it never completed.
__device__ __forceinline__ bool tc5_mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tc5_tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace qc
