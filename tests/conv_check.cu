// Check of the integer-arithmetic conversions of the device helpers (d2f:
// binary64 -> binary32 round-to-nearest-even, i2d: int -> binary64) against
// the hardware conversions, bit for bit, over random and edge-case inputs.
// Built and run by test_conversions.py; prints "mismatches <n>" and exits 0
// when there are none.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "dmr_device.cuh"

using namespace dmr;

__device__ unsigned long long mix64(unsigned long long z) {
  // SplitMix64 finaliser
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Input k: the exponent field drawn from [880, 1165] (both ends of the normal
// binary32 range and beyond) for 7 in 8 inputs, any exponent otherwise; the
// 29 dropped fraction bits forced to a tie, or to one above or below it, for
// some inputs; a few fixed specials.
__device__ double input(unsigned long long k) {
  const unsigned long long r = mix64(k), r2 = mix64(k ^ 0x5555555555555555ull);
  unsigned long long bits = r;
  if ((r2 & 7) != 0) {
    const unsigned long long ex = 880 + (r2 >> 8) % 286;
    bits = (r & 0x800fffffffffffffull) | (ex << 52);
  }
  switch ((r2 >> 4) & 15) {
    case 0: bits = (bits & ~0x1fffffffull) | 0x10000000ull; break;
    case 1: bits = (bits & ~0x1fffffffull) | 0x0fffffffull; break;
    case 2: bits = (bits & ~0x1fffffffull) | 0x10000001ull; break;
    case 3: bits |= 0x000fffffe0000000ull | 0x10000000ull; break;  // all-ones kept fraction: carry
    default: break;
  }
  const unsigned long long special[10] = {0x0ull, 0x8000000000000000ull, 0x7ff0000000000000ull,
                                          0xfff0000000000000ull, 0x7ff8000000000000ull, 0x0000000000000001ull,
                                          0x47efffffe0000000ull, 0x47effffff0000000ull, 0x3810000000000000ull,
                                          0x380fffffffffffffull};
  if (k < 10) bits = special[k];
  return __longlong_as_double((long long)bits);
}

__global__ void k_check(unsigned long long n, unsigned long long* bad, unsigned long long* first) {
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const double x = input(k);
    const float a = d2f(x), b = __double2float_rn(x);
    const bool same = __float_as_uint(a) == __float_as_uint(b) || (a != a && b != b);
    if (!same) {
      atomicAdd(bad, 1ull);
      atomicCAS(first, ~0ull, (unsigned long long)__double_as_longlong(x));
    }
    const int v = (int)(unsigned)mix64(k * 3 + 1) >> (int)(k & 31);
    const int vs[4] = {0, 1, -1, (int)0x80000000u};
    const int w = k < 4 ? vs[k] : (k < 8 ? 0x7fffffff - (int)(k - 4) : v);
    if (__double_as_longlong(i2d(w)) != __double_as_longlong((double)w)) atomicAdd(bad + 1, 1ull);
  }
}

int main() {
  unsigned long long *bad, *first;
  cudaMalloc(&bad, 2 * sizeof(unsigned long long));
  cudaMalloc(&first, sizeof(unsigned long long));
  cudaMemset(bad, 0, 2 * sizeof(unsigned long long));
  cudaMemset(first, 0xff, sizeof(unsigned long long));
  const unsigned long long n = 1ull << 28;
  k_check<<<1024, 256>>>(n, bad, first);
  unsigned long long h[2] = {0, 0}, f = 0;
  cudaError_t e = cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost);
  cudaMemcpy(&f, first, sizeof(f), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    printf("cuda error %s\n", cudaGetErrorString(e));
    return 2;
  }
  printf("inputs %llu d2f mismatches %llu i2d mismatches %llu first %016llx\n", n, h[0], h[1], f);
  printf("mismatches %llu\n", h[0] + h[1]);
  return (h[0] + h[1]) == 0 ? 0 : 1;
}
