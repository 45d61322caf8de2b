// Residue-number (CRT) emulation of FP64 matrix products on BF16 tensor cores.
//
// C = op(A) op(B), each operand row (of op(A)) / column (of op(B)) scaled by a
// power of two and rounded to a signed integer of at most beta bits; the
// integer product is then known modulo each of n pairwise-coprime moduli
// p_j <= 128 from n BF16 products of the balanced residues (|residue| <= 64,
// so every partial sum of K <= 4096 products is an integer of magnitude
// <= 4096 * 64 * 64 = 2^24 and the FP32 accumulation is exact), and is
// recovered exactly by the Chinese remainder theorem as long as
// 2 K 2^(2 beta) < prod p_j.  (Ozaki, Uchino, Imamura, "Ozaki Scheme II: A
// GEMM-oriented emulation of floating-point matrix multiplication using an
// integer modular technique", 2024.)
#pragma once

#include <cstdint>

namespace cpinv {
namespace crt {

constexpr int kMaxMod = 24;
// Pairwise coprime, largest first: 2^7, 127, 5^3, 11^2, 7*17, 9*13, then primes.
constexpr int kModuli[kMaxMod] = {128, 127, 125, 121, 119, 117, 113, 109, 107, 103, 101, 97,
                                  89,  83,  79,  73,  71,  67,  61,  59,  53,  47,  43,  41};
constexpr int kLimbs = 5;  // 32-bit limbs of the CRT sums (< 2^160)

// kModuli[j], usable in device code (constant-folds for a constant j)
__host__ __device__ constexpr int modulus(int j) {
  return j == 0 ? 128 : j == 1 ? 127 : j == 2 ? 125 : j == 3 ? 121 : j == 4 ? 119 : j == 5 ? 117
       : j == 6 ? 113 : j == 7 ? 109 : j == 8 ? 107 : j == 9 ? 103 : j == 10 ? 101 : j == 11 ? 97
       : j == 12 ? 89 : j == 13 ? 83 : j == 14 ? 79 : j == 15 ? 73 : j == 16 ? 71 : j == 17 ? 67
       : j == 18 ? 61 : j == 19 ? 59 : j == 20 ? 53 : j == 21 ? 47 : j == 22 ? 43 : 41;
}

// Constants of the first n moduli (host-computed, passed by value to kernels).
struct Consts {
  int32_t n;
  int32_t shift;                   // bit position used for the quotient estimate
  float inv_ptop;                  // 1 / float(P >> shift)
  int32_t pad;
  uint32_t P[kLimbs];              // P = prod p_j
  uint32_t halfP[kLimbs];          // floor(P / 2)
  uint32_t Mj[kMaxMod][kLimbs];    // P / p_j
  uint8_t tab[kMaxMod][128];       // tab[j][r] = (r * y_j) mod p_j, y_j = (P/p_j)^-1 mod p_j
};

// Smallest n whose modulus product exceeds 2^bits (bits < 155), or -1.
int moduli_for_bits(int bits);
// Fills c for the first n moduli.
void make_consts(int n, Consts* c);

}  // namespace crt
}  // namespace cpinv
