// snn_device.cuh -- device helpers shared by the kernels of the library.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace snn {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds; each multiplies words 0 and 2 by the
// two round constants, xors the high halves into the other words and the key,
// and permutes; the key advances by the Weyl constants after every round.
// Counter = (a, b, stream tag, 0), key = 64-bit seed.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Uniform integer in [0, n): (x * n) >> 32.
__device__ __forceinline__ uint32_t below(uint32_t x, uint32_t n) {
  return __umulhi(x, n);
}

__device__ __forceinline__ uint32_t lane_id() {
  uint32_t l;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}

// Periodic wrap of a coordinate that may lie several periods outside [0, n).
__device__ __forceinline__ int wrap(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

}  // namespace snn
