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

// Balanced residues (|v| <= 64) of the signed integer (neg ? -a : a), a <
// 2^63, modulo the first n_mod moduli, as BF16 at o[j * plane].  a is cut
// into 21-bit chunks once; each residue is then one reduction of a value
// below 2^29.
__device__ __forceinline__ void store_residues(uint64_t a, bool neg, int n_mod, __nv_bfloat16* o,
                                               size_t plane) {
  const uint32_t a0 = (uint32_t)(a & 0x1FFFFF), a1 = (uint32_t)((a >> 21) & 0x1FFFFF),
                 a2 = (uint32_t)(a >> 42);
#pragma unroll
  for (int j = 0; j < kMaxMod; ++j) {
    if (j >= n_mod) break;
    const uint32_t p = (uint32_t)modulus(j);
    const uint32_t c1 = (uint32_t)((1ull << 21) % p), c2 = (uint32_t)((1ull << 42) % p);
    const uint32_t h = (p - 1) / 2;
    // v = ((a + h) mod p) - h, |v| <= 64; the residue of -a is -v
    const uint32_t r = (a2 * c2 + a1 * c1 + a0 + h) % p;
    const float f = __int_as_float((int)(0x4B400000u - h) + (int)r) - 12582912.0f;
    const unsigned short bits = (unsigned short)((__float_as_uint(f) >> 16) ^ (neg ? 0x8000u : 0u));
    o[j * plane] = __ushort_as_bfloat16(bits);
  }
}

// The balanced residues of two integers modulo the J-th modulus as BF16
// bits packed two per word (the first in the low half): a, b < 2^63 given by
// their three 21-bit chunks, the signs in sgn (0x8000 for a negative first,
// 0x80000000 for a negative second).  With h = (p - 1) / 2 the balanced
// residue of a is v = ((a + h) mod p) - h (|v| <= 64), one reduction of a
// value below 2^29; the offset h rides in the sum and in the FP32 constant
// that turns r - h into its float, whose top 16 bits are its BF16 bits (an
// integer of at most 7 bits is exact in BF16); the residue of -a is -v, a
// sign flip of those bits.
template <int J>
__device__ __forceinline__ uint32_t residue_pair_bf16(uint32_t a0, uint32_t a1, uint32_t a2,
                                                      uint32_t b0, uint32_t b1, uint32_t b2,
                                                      uint32_t sgn) {
  constexpr uint32_t p = (uint32_t)modulus(J);
  constexpr uint32_t c1 = (uint32_t)((1ull << 21) % p);
  constexpr uint32_t c2 = (uint32_t)((1ull << 42) % p);
  constexpr uint32_t h = (p - 1) / 2;
  const uint32_t ra = (a2 * c2 + a1 * c1 + a0 + h) % p;
  const uint32_t rb = (b2 * c2 + b1 * c1 + b0 + h) % p;
  const float fa = __int_as_float((int)(0x4B400000u - h) + (int)ra) - 12582912.0f;
  const float fb = __int_as_float((int)(0x4B400000u - h) + (int)rb) - 12582912.0f;
  return __byte_perm(__float_as_uint(fa), __float_as_uint(fb), 0x7632) ^ sgn;
}



// ---------------------------------------------------------------------------
// CRT reconstruction: exact integer (5 x 32-bit limbs) -> FP64
// ---------------------------------------------------------------------------

// +-mant * 2^e outside the normal exponent range: the FP64 unit handles the
// under/overflow; out of line, so that the common path never executes it.
__device__ __noinline__ inline double compose_out_of_range(bool neg, uint64_t mant, int e) {
  const double d = ldexp((double)mant, e);
  return neg ? -d : d;
}

__device__ __forceinline__ double compose_double(bool neg, const uint32_t (&mag)[crt::kLimbs],
                                                 int scale) {
  // correctly rounded mag * 2^scale (mag < 2^160), via integer operations
  int top = -1;
#pragma unroll
  for (int i = crt::kLimbs - 1; i >= 0; --i)
    if (top < 0 && mag[i]) top = 32 * i + 31 - __clz(mag[i]);
  if (top < 0) return neg ? -0.0 : 0.0;
  // 64 bits starting at bit (top - 63), sticky below
  const int lo_bit = top - 63;
  uint64_t t = 0;
  bool sticky = false;
#pragma unroll
  for (int i = 0; i < crt::kLimbs; ++i) {
    const int base = 32 * i;  // bits base .. base+31 of mag
    const uint64_t w = mag[i];
    const int off = base - lo_bit;  // where bit `base` lands in t
    if (off >= 64 || off <= -32) {
      if (off <= -32 && w) sticky = true;
      continue;
    }
    if (off >= 0) t |= w << off;
    else {
      t |= w >> (-off);
      if (w & ((1ull << (-off)) - 1ull)) sticky = true;
    }
  }
  uint64_t mant = t >> 11;
  const uint64_t rem = t & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (sticky || (mant & 1ull)))) ++mant;
  int e = top;  // value = mant * 2^(top - 52)
  if (mant >> 53) {
    mant >>= 1;
    ++e;
  }
  const int biased = e + scale + 1023;
  if (biased <= 0 || biased >= 2047) return compose_out_of_range(neg, mant, e - 52 + scale);
  const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)biased << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// select S[k] for a uniform runtime k without local memory
__device__ __forceinline__ uint32_t limb_at(const uint32_t (&S)[crt::kLimbs], int k) {
  uint32_t w = 0;
#pragma unroll
  for (int l = 0; l < crt::kLimbs; ++l) w = (l == k) ? S[l] : w;
  return w;
}

struct CrtShared {
  uint8_t tab[crt::kMaxMod][128];
  uint32_t Mj[crt::kMaxMod][crt::kLimbs];
  uint32_t P[crt::kLimbs];
  uint32_t halfP[crt::kLimbs];
};

// S (the CRT sum, < n P) -> X = S mod P centred into (-P/2, P/2], as a
// two's complement integer of kLimbs limbs.
__device__ __forceinline__ void crt_centre(const uint32_t (&S)[crt::kLimbs], const uint32_t* P,
                                           const uint32_t* halfP, int shift, float inv_ptop,
                                           uint32_t (&Y)[crt::kLimbs]) {
  // q = floor(S / P) in [0, n): estimate from the top bits, then correct
  uint64_t stop = 0;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int pos = shift + 32 * b;  // 32-bit chunk of S >> shift
    const int li = pos >> 5, off = pos & 31;
    uint32_t w = limb_at(S, li) >> off;
    if (off) w |= limb_at(S, li + 1) << (32 - off);
    stop |= (uint64_t)w << (32 * b);
  }
  // from the top 32 bits of the window (stop < 2^63): a 64-bit integer to
  // float conversion would run on the FP64 pipe
  int qe = (int)floorf((float)(uint32_t)(stop >> 32) * (inv_ptop * 4294967296.0f));
  qe = qe < 0 ? 0 : qe;
  // X = S - qe * P  (signed, two's complement over the limbs)
  int64_t borrow = 0;
  uint32_t X[crt::kLimbs];
#pragma unroll
  for (int l = 0; l < crt::kLimbs; ++l) {
    const int64_t v = (int64_t)S[l] - (int64_t)((uint64_t)qe * P[l]) + borrow;
    X[l] = (uint32_t)v;
    borrow = v >> 32;  // arithmetic
  }
  // fix-up: bring X into [0, P) (the estimate is off by at most one)
#pragma unroll
  for (int pass = 0; pass < 1; ++pass) {
    if ((int32_t)X[crt::kLimbs - 1] < 0) {  // X < 0: X += P
      uint64_t cc = 0;
#pragma unroll
      for (int l = 0; l < crt::kLimbs; ++l) {
        const uint64_t v = (uint64_t)X[l] + P[l] + cc;
        X[l] = (uint32_t)v;
        cc = v >> 32;
      }
    } else {
      bool ge = true, decided = false;  // X >= P ?
#pragma unroll
      for (int l = crt::kLimbs - 1; l >= 0; --l) {
        if (!decided && X[l] != P[l]) {
          ge = X[l] > P[l];
          decided = true;
        }
      }
      if (ge) {
        int64_t bb = 0;
#pragma unroll
        for (int l = 0; l < crt::kLimbs; ++l) {
          const int64_t v = (int64_t)X[l] - (int64_t)P[l] + bb;
          X[l] = (uint32_t)v;
          bb = v >> 32;
        }
      }
    }
  }
  // centre: X > P/2 -> X - P (negative, two's complement)
  bool gt = false, decided = false;
#pragma unroll
  for (int l = crt::kLimbs - 1; l >= 0; --l) {
    if (!decided && X[l] != halfP[l]) {
      gt = X[l] > halfP[l];
      decided = true;
    }
  }
  int64_t bb = 0;
#pragma unroll
  for (int l = 0; l < crt::kLimbs; ++l) {
    const int64_t v = (int64_t)X[l] - (int64_t)P[l] + bb;
    Y[l] = gt ? (uint32_t)v : X[l];
    bb = v >> 32;
  }
}

// A two's complement integer of kLimbs limbs times 2^scale, correctly
// rounded to FP64.
__device__ __forceinline__ double limbs_to_double(const uint32_t (&Y)[crt::kLimbs], int scale) {
  const bool neg = (int32_t)Y[crt::kLimbs - 1] < 0;
  uint32_t mag[crt::kLimbs];
  uint64_t c = 1;
#pragma unroll
  for (int l = 0; l < crt::kLimbs; ++l) {
    if (neg) {
      const uint64_t v = (uint64_t)(~Y[l]) + c;
      mag[l] = (uint32_t)v;
      c = v >> 32;
    } else {
      mag[l] = Y[l];
    }
  }
  return compose_double(neg, mag, scale);
}

// Y += (hi:lo), a signed 128-bit two's complement integer.
__device__ __forceinline__ void limbs_add128(uint32_t (&Y)[crt::kLimbs], uint64_t lo, int64_t hi) {
  const uint32_t ext = hi < 0 ? 0xFFFFFFFFu : 0u;
  const uint32_t w[crt::kLimbs] = {(uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)(uint64_t)hi,
                                   (uint32_t)((uint64_t)hi >> 32), ext};
  uint64_t c = 0;
#pragma unroll
  for (int l = 0; l < crt::kLimbs; ++l) {
    const uint64_t v = (uint64_t)Y[l] + w[l] + c;
    Y[l] = (uint32_t)v;
    c = v >> 32;
  }
}

// S (the CRT sum, < n P) -> centred X = S mod P in (-P/2, P/2] -> FP64,
// correctly rounded, times 2^scale.
__device__ __forceinline__ double crt_finish(const uint32_t (&S)[crt::kLimbs],
                                             const uint32_t* P, const uint32_t* halfP, int shift,
                                             float inv_ptop, int scale) {
  uint32_t Y[crt::kLimbs];
  crt_centre(S, P, halfP, shift, inv_ptop, Y);
  return limbs_to_double(Y, scale);
}

}  // namespace crt
}  // namespace cpinv
