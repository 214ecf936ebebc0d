// fixed_point.cuh -- the integer rule of the deposit (Eq. smooth with the
// lookup table of Sect. 3.1), shared by every deposit kernel of the library.
#pragma once
#include <cstdint>

namespace parts {

// Integer rule of one tap. Axis weights W (2^-24 units) come from the table;
// the mass significand is folded into the x weights, MX = (Wx msig + 2^15) >> 16;
// the y and z weights are combined per row, R = (Wy Wz + 2^15) >> 16; the
// contribution is the exact product P = R MX shifted to 2^-Kacc mass units
// with round-half-up (sh = 40 - Kacc - e2, |m| = msig 2^e2).
__device__ __forceinline__ uint32_t fold_x(uint32_t wx, uint32_t msig) {
  return (uint32_t)(((uint64_t)wx * msig + 32768ull) >> 16);
}
__device__ __forceinline__ uint32_t row_yz(uint32_t wy, uint32_t wz) {
  return (uint32_t)(((uint64_t)wy * wz + 32768ull) >> 16);
}
__device__ __forceinline__ uint64_t round_shift(uint64_t p, int sh) {
  if (p == 0) return 0;
  if (sh <= 0) return p << (-sh);
  if (sh >= 64) return 0;
  return (p + (1ull << (sh - 1))) >> sh;
}
// The same rule from the three axis weights (for kernels that do not keep the
// per-particle tables).
__device__ __forceinline__ uint64_t tap_contrib(uint32_t wx, uint32_t wy, uint32_t wz, uint32_t msig, int sh) {
  return round_shift((uint64_t)row_yz(wy, wz) * fold_x(wx, msig), sh);
}

// FP32 mass -> (significand, power of two): |m| = msig * 2^e2.
__device__ __forceinline__ void mass_parts(uint32_t mb, uint32_t* msig, int* e2) {
  int eb = (mb >> 23) & 0xFF;
  *msig = eb ? ((mb & 0x7FFFFFu) | 0x800000u) : (mb & 0x7FFFFFu);
  *e2 = eb ? eb - 150 : -149;
}

}  // namespace parts
