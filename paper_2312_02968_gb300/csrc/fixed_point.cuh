// fixed_point.cuh -- the integer rule of the deposit (Eq. smooth with the
// lookup table of Sect. 3.1), shared by every deposit kernel of the library.
#pragma once
#include <cstdint>

namespace parts {

// One tap: 2^-24 axis weights -> w3 in 2^-40 units (two round-half-up
// narrowings) -> times the mass significand -> 2^-Kacc units (round half up).
__device__ __forceinline__ uint64_t tap_contrib(uint32_t wx, uint32_t wy, uint32_t wz, uint32_t msig, int sh) {
  uint64_t wxy = (uint64_t)wx * (uint64_t)wy;
  uint64_t wxy16 = (wxy + 32768ull) >> 16;
  uint64_t w3 = (wxy16 * (uint64_t)wz + 32768ull) >> 16;
  uint64_t p = w3 * (uint64_t)msig;
  if (p == 0) return 0;
  if (sh <= 0) return p << (-sh);
  if (sh >= 64) return 0;
  return (p + (1ull << (sh - 1))) >> sh;
}

// FP32 mass -> (significand, power of two): |m| = msig * 2^e2.
__device__ __forceinline__ void mass_parts(uint32_t mb, uint32_t* msig, int* e2) {
  int eb = (mb >> 23) & 0xFF;
  *msig = eb ? ((mb & 0x7FFFFFu) | 0x800000u) : (mb & 0x7FFFFFu);
  *e2 = eb ? eb - 150 : -149;
}

}  // namespace parts
