// Device helpers shared by the kernels that write residue planes.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "crt.h"

namespace cpinv {
namespace crt {

// |x| * 2^(beta - e) rounded to nearest, as an unsigned magnitude, where the
// row bound is |x| < 2^e with e = Emax - 1022 (Emax a biased exponent):
//   a = m * 2^(E - Emax + beta - 53)   (m the 53-bit significand of x).
// With Emax at least the biased exponent of every |x| in the row, a < 2^beta.
__device__ __forceinline__ uint64_t integerize(uint64_t b, int Emax, int beta) {
  const int E = (int)((b >> 52) & 0x7FF);
  if ((b << 1) == 0 || Emax == 0) return 0;
  uint64_t m = b & 0xFFFFFFFFFFFFFull;
  int Eeff = E;
  if (E == 0) Eeff = 1;
  else m |= 0x10000000000000ull;
  const int sh = Eeff - Emax + beta - 53;
  if (sh >= 0) return m << sh;  // beta <= 62 keeps this below 2^63
  const int rs = -sh;
  if (rs > 63) return 0;
  const uint64_t half = (uint64_t)1 << (rs - 1);
  return (m + half) >> rs;
}

// Balanced residues (|v| <= 64) of the signed integer (neg ? -a : a) modulo
// the first n_mod moduli, as BF16 at o[j * plane].
__device__ __forceinline__ void store_residues(uint64_t a, bool neg, int n_mod, __nv_bfloat16* o,
                                               size_t plane) {
  const uint32_t ahi = (uint32_t)(a >> 32), alo = (uint32_t)a;
#pragma unroll
  for (int j = 0; j < kMaxMod; ++j) {
    if (j >= n_mod) break;
    const uint32_t p = (uint32_t)modulus(j);
    const uint32_t two32 = (uint32_t)((((uint64_t)1) << 32) % p);
    uint32_t r = ((ahi % p) * two32 + (alo % p)) % p;
    if (neg && r) r = p - r;
    const int v = (int)r > (int)(p / 2) ? (int)r - (int)p : (int)r;
    o[j * plane] = __float2bfloat16_rn((float)v);
  }
}

// BF16 bits of a small integer |v| <= 64 (exact): the float with those bits is
// formed by adding v to 1.5 * 2^23 in the integer domain and subtracting it
// back in FP32 (exact), and its top 16 bits are the BF16 encoding.
__device__ __forceinline__ uint32_t small_int_bf16_bits(int v) {
  const float f = __int_as_float(0x4B400000 + v) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

// Balanced residue of (neg ? -a : a) modulo the j-th modulus, from the three
// 21-bit chunks of a < 2^63 (one reduction of a value below 2^29).
template <int J>
__device__ __forceinline__ int residue21(uint32_t a0, uint32_t a1, uint32_t a2, bool neg) {
  constexpr uint32_t p = (uint32_t)modulus(J);
  constexpr uint32_t c1 = (uint32_t)((1ull << 21) % p);
  constexpr uint32_t c2 = (uint32_t)((1ull << 42) % p);
  uint32_t r = (a2 * c2 + a1 * c1 + a0) % p;
  if (neg && r) r = p - r;
  return (int)r > (int)(p / 2) ? (int)r - (int)p : (int)r;
}

}  // namespace crt
}  // namespace cpinv
