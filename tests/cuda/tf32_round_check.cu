// Checks the library's integer TF32 rounding (warp_mma.h) against the
// hardware conversion cvt.rna.tf32.f32 on every 32-bit pattern that is not a
// NaN, and the split a = big + small on a sample.  Prints the mismatch counts;
// exits 0 when both are zero.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "warp_mma.h"

__global__ void k_check(unsigned long long* bad_round, unsigned long long* bad_split) {
  const uint64_t n = 1ull << 32;
  unsigned long long br = 0, bs = 0;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t u = (uint32_t)e;
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu) != 0u) continue;  // NaN
    const float x = __uint_as_float(u);
    uint32_t hw;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hw) : "f"(x));
    if (fno::wm::tf32_rna_bits(x) != hw) ++br;
    if ((u & 0xfffu) == 0x5a5u && (u & 0x7f800000u) < 0x7f000000u) {
      uint32_t big, small;
      fno::wm::tf32_split(x, big, small);
      // big and small are TF32 values and big + small reproduces x to TF32 of the residual
      if ((big & 0x1fffu) != 0u || (small & 0x1fffu) != 0u) ++bs;
      const float r = x - __uint_as_float(big);
      uint32_t hs;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hs) : "f"(r));
      if (hs != small) ++bs;
    }
  }
  atomicAdd(bad_round, br);
  atomicAdd(bad_split, bs);
}

int main() {
  unsigned long long* d;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return 2;
  cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  k_check<<<1024, 256>>>(d, d + 1);
  if (cudaDeviceSynchronize() != cudaSuccess) return 2;
  unsigned long long h[2];
  cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  printf("round mismatches %llu split mismatches %llu\n", h[0], h[1]);
  return (h[0] == 0 && h[1] == 0) ? 0 : 1;
}
