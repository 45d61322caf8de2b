// Device-side pieces of the full-rank Cholesky shared by the FP64 kernels
// (chol.cu) and the exact-slice panel kernel (chol_exact.cu): the pivot's
// 1/sqrt and the four-warp factorisation of a diagonal block.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace cpinv {
namespace chol {

// Seed y0 ~ 1/sqrt(d) (about 22 correct bits) for a finite d > 0 given by
// its bit pattern, with integer operations only (FP64 <-> FP32 conversions
// and FP64 instructions are slow on this part): d = 2^(2k) f with f in
// [1, 4) taken to float by truncating its significand, y0 = 2^-k rsqrtf(f).
// A subnormal d is normalised by a leading-zero count first.
__device__ __forceinline__ double rsqrt_seed(uint64_t bits) {
  const int ex = (int)((bits >> 52) & 0x7FF);
  const uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
  const bool sub = ex == 0;
  const int sh = sub ? __clzll((long long)mant) - 11 : 0;
  const int E = sub ? -1022 - sh : ex - 1023;  // d = 1.frac 2^E
  const uint64_t frac = (mant << sh) & 0xFFFFFFFFFFFFFull;
  const int k = E >> 1;  // floor(E / 2)
  const uint32_t fbits = ((uint32_t)(127 + (E - 2 * k)) << 23) | (uint32_t)(frac >> 29);
  const uint32_t sb = __float_as_uint(rsqrtf(__uint_as_float(fbits)));
  const int es = (int)((sb >> 23) & 0xFF) - 127 - k;  // exponent of the seed
  return __longlong_as_double(
      (long long)(((uint64_t)(es + 1023) << 52) | ((uint64_t)(sb & 0x7FFFFF) << 29)));
}

// One third-order correction of the seed: with e = 1 - d y0^2,
//   1/sqrt(d) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + O(e^3)),
// accurate to O(e^3) ~ 2^-66.  e is formed as 1 - (d y0) y0, which stays in
// range for subnormal and huge d.  The pivot's column is scaled by the same
// series, x / sqrt(d) = s + (s e)(1/2 + 3e/8) with s = x y0, so the product
// x y0 runs beside the correction instead of after it.
__device__ __forceinline__ double rsqrt_e(double d, double y0) { return fma(-(d * y0), y0, 1.0); }
__device__ __forceinline__ double rsqrt_apply(double x, double y0, double e) {
  const double s = x * y0;
  return fma(s * e, fma(e, 0.375, 0.5), s);
}

// Named barriers 1 and 2 (0 is __syncthreads): producer / consumer hand-off
// of one column between the four warps of the diagonal-block kernel.
__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

constexpr int kDiagWarps = 4;
constexpr int kDiagThreads = 32 * kDiagWarps;

// Factorisation of the diagonal block of panel k0 (b <= 32) by one CTA of
// four warps.  Lane i holds row i; warp w holds the columns j = w (mod 4).
// Column c is finished by its owner warp (pivot test, square root, scaling)
// and handed to the others through a triple-buffered shared column and a
// named barrier: the owner arrives, the others wait.  Look-ahead: the owner
// of column c+1 applies the update of column c to that column first and
// finishes it before its other updates, so the hand-off of every column
// waits for one update and one pivot only.  The columns are processed in
// groups of four (one per warp); after each group every warp's registers
// shift by one column, so register indices stay compile-time constants in a
// loop that is not unrolled (a fully unrolled factorisation is long enough
// to stall on instruction fetch).  The sequence of operations on every entry
// (updates in column order, the pivot, the scaling) is that of the plain
// column-by-column algorithm.
__device__ __forceinline__ void diag_chol_block(double* A, int64_t lda, Dim nd, int64_t k0, int b,
                                                DevState* st, const int64_t* rdev,
                                                uint8_t* accepted, double* dinv, int spd) {
  const int64_t n = eval_dim(nd, rdev);
  if (k0 >= n) return;
  const int bw = (int)((n - k0) < b ? (n - k0) : b);
  __shared__ double colbuf[3][32];
  __shared__ double y0_s[32], e_s[32];
  __shared__ int acc_s[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // the pivot test d > tol on the bit patterns (tol >= 0: a negative d, -0
  // and NaN compare below or are excluded; +inf passes as it does in FP64)
  const long long tolbits = __double_as_longlong(spd ? 0.0 : st->tol);
  // a[q]: this lane's entry of column 4 (t + q) + w during group t
  double a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = w + kDiagWarps * q;
    // L2 loads: other CTAs of a fused launch may have just written the block
    a[q] = (lane < bw && j < bw && j <= lane) ? __ldcg(A + (k0 + lane) * lda + (k0 + j)) : 0.0;
  }
  // Finishes column c held in `acol` (owner warp only); returns L(lane, c).
  // Lane c's entry d is broadcast first and every lane runs the pivot test
  // and the 1/sqrt chain on it (uniform: no divergence, no broadcast after
  // the chain); a rejected pivot gives a zero column.
  auto pivot = [&](int c, double acol) -> double {
    const double d = __shfl_sync(0xffffffffu, acol, c);
    const long long db = __double_as_longlong(d);
    const bool ok = db > tolbits && db <= 0x7FF0000000000000ll;
    const double y0 = rsqrt_seed((uint64_t)db);
    const double e = rsqrt_e(d, y0);
    const double lv = rsqrt_apply(acol, y0, e);  // lane c: d / sqrt(d)
    const double l = (ok && lane >= c) ? lv : 0.0;
    colbuf[c % 3][lane] = l;
    if (lane == c) {
      acc_s[c] = ok;
      y0_s[c] = y0;
      e_s[c] = e;
    }
    return l;
  };
  if (w == 0) {
    a[0] = pivot(0, a[0]);
    __syncwarp();
    __threadfence_block();
    bar_arrive(1, kDiagThreads);
  }
#pragma unroll 1
  for (int t = 0; kDiagWarps * t < bw; ++t) {
#pragma unroll
    for (int u = 0; u < kDiagWarps; ++u) {
      const int c = kDiagWarps * t + u;
      if (c >= bw) break;
      const int buf = c % 3;
      if (w != u) bar_sync(1 + (c & 1), kDiagThreads);
      else __syncwarp();
      const double li = colbuf[buf][lane];
      const int nxt = c + 1;
      // the owner of column c+1 is warp (u+1) mod 4; the column is its a[0]
      // within this group, its a[1] when it opens the next group
      const int qn = (u + 1 < kDiagWarps) ? 0 : 1;
      const bool ahead = nxt < bw && w == ((u + 1) & (kDiagWarps - 1));
      if (ahead) {
        if (lane >= nxt) a[qn] = fma(-li, colbuf[buf][nxt], a[qn]);
        a[qn] = pivot(nxt, a[qn]);
        __syncwarp();
        __threadfence_block();
        bar_arrive(1 + (nxt & 1), kDiagThreads);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q == 0 && w <= u) continue;  // column 4t + w is not after c
        if (ahead && q == qn) continue;
        const int j = kDiagWarps * (t + q) + w;
        if (j < bw && lane >= j) a[q] = fma(-li, colbuf[buf][j], a[q]);
      }
    }
    // column 4t + w is final: store it, then shift the registers by one column
    const int j0 = kDiagWarps * t + w;
    if (j0 < bw && lane < bw && lane >= j0) A[(k0 + lane) * lda + (k0 + j0)] = a[0];
#pragma unroll
    for (int q = 0; q < 7; ++q) a[q] = a[q + 1];
    a[7] = 0.0;
  }
  bar_sync(3, kDiagThreads);  // the four warps only (the caller's CTA may be larger)
  if (threadIdx.x < bw) {
    // 1/T(c, c) from the stored seed and correction, all columns at once
    const int c = threadIdx.x;
    const double y0 = y0_s[c], e = e_s[c];
    dinv[c] = acc_s[c] ? fma(y0 * e, fma(e, 0.375, 0.5), y0) : 0.0;
    if (!spd && accepted) accepted[k0 + threadIdx.x] = (uint8_t)acc_s[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    int kept = 0;
    for (int c = 0; c < bw; ++c) kept += acc_s[c];
    if (spd) {
      if (kept != bw) atomicOr(&st->status, ST_NUMERICAL);
      atomicAdd((unsigned long long*)&st->rank_n, (unsigned long long)kept);
    }
  }
}

}  // namespace chol
}  // namespace cpinv
