// split_common.cuh -- pieces shared by the two split-precision tensor-core apply kernels
// (destination-stationary in apply_split.cu, source-stationary in apply_src.cu): the
// shared-memory operand layout the MMAs read, the BF16 piece split, and warpgroup barriers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mra {
namespace split {

constexpr int MG_BYTES = 272;           // stride of the 8-row groups: 256 B of core matrices + 16 B
                                        // so that consecutive groups start 4 banks apart
constexpr int TILE_BYTES = 16 * MG_BYTES;  // one 128 x 16 BF16 operand tile
constexpr int BPIECE_BYTES = 512;       // one 16 x 16 BF16 block piece
constexpr int BSTAGE_BYTES = 3 * BPIECE_BYTES;  // the three pieces of one block
constexpr long long WAIT_CYCLES = 4000000000LL;  // bounded mbarrier wait (~2 s)

// byte offset of element (row m, contraction kk) in an MN-major operand: core
// matrices of 8 contraction rows x 8 consecutive rows (128 B); the two
// contraction groups of a row group 128 B apart (descriptor LBO), the 16 row
// groups of a 128-row tile MG_BYTES apart (descriptor SBO)
__device__ __forceinline__ uint32_t a_off(int m, int kk) {
  return (uint32_t)((m >> 7) * TILE_BYTES + ((m & 127) >> 3) * MG_BYTES + (kk >> 3) * 128 +
                    (kk & 7) * 16 + (m & 7) * 2);
}

// x (FP64) as three BF16 pieces, x = p0 + p1 + p2 to 24 bits
__device__ __forceinline__ void split3(double x, __nv_bfloat16 &p0, __nv_bfloat16 &p1,
                                       __nv_bfloat16 &p2) {
  p0 = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(p0);
  p1 = __double2bfloat16(r);
  r -= (double)__bfloat162float(p1);
  p2 = __double2bfloat16(r);
}

// Split x and y into three BF16 pieces each (x = x0 + x1 + x2 to 24 bits), packed in pairs.
__device__ __forceinline__ void split_pair(float x, float y, __nv_bfloat162 &h0, __nv_bfloat162 &h1,
                                           __nv_bfloat162 &h2) {
  h0 = __floats2bfloat162_rn(x, y);
  float2 f0 = __bfloat1622float2(h0);
  float rx = x - f0.x, ry = y - f0.y;
  h1 = __floats2bfloat162_rn(rx, ry);
  float2 f1 = __bfloat1622float2(h1);
  h2 = __floats2bfloat162_rn(rx - f1.x, ry - f1.y);
}

// Named barrier over one warpgroup (128 threads) with an OR vote.
__device__ __forceinline__ bool wg_vote_or(int barrier_id, bool flag) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)flag), "r"(barrier_id)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void wg_sync(int barrier_id) {
  asm volatile("bar.sync %0, 128;" ::"r"(barrier_id) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void st_shared32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_shared128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

}  // namespace split
}  // namespace mra
