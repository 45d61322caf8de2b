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
// x y0 runs beside the correction instead of after it.  (Squaring the seed
// exactly in the integer unit saves one FP64 instruction but measured
// slower: the range test and the integer chain cost more than it saves.)
__device__ __forceinline__ double rsqrt_e(double d, double y0) { return fma(-(d * y0), y0, 1.0); }
__device__ __forceinline__ double rsqrt_apply(double x, double y0, double e) {
  const double s = x * y0;
  return fma(s * e, fma(e, 0.375, 0.5), s);
}

// Named barrier 3 (0 is __syncthreads) joins the four warps of the
// diagonal-block factorisation inside a larger CTA.
__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Column hand-off: one shared-memory barrier per column, completed by the 32
// arrivals of the owner warp's lanes (each after writing its entry; arrive
// has release semantics) and waited on by every other warp on its own
// (acquire), so a warp still issuing its updates never holds back the next
// pivot.  The wait is bounded: false after kColSpinLimit polls.
constexpr uint32_t kColSpinLimit = 1u << 22;
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void col_init(uint64_t* mb, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void col_inval(uint64_t* mb) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(mb)) : "memory");
}
__device__ __forceinline__ void col_publish(uint64_t* mb) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mb)) : "memory");
}
__device__ __forceinline__ bool col_wait(uint64_t* mb) {
  for (uint32_t it = 0; it < kColSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(mb))
        : "memory");
    if (ok) return true;
  }
  return false;
}

constexpr int kDiagWarps = 4;
constexpr int kDiagThreads = 32 * kDiagWarps;

// Shared memory of a diagonal-block factorisation, supplied by the calling
// kernel (which may alias it with memory its other phases use).
struct DiagScratch {
  double col[32][32];  // col[c][i]: L(i, c), the finished column c
  uint64_t bar[32];    // per-column hand-off barriers
  double y0[32];       // seed and correction of 1/sqrt of each pivot
  double e[32];
  int acc[32];         // kept flags
};

// Factorisation of the diagonal block of panel k0 (b <= 32) by one CTA of
// four warps.  Lane i holds row i; warp w holds the columns
// j = w (mod 4).  Column c is finished by its owner warp (pivot test, square
// root, scaling) and handed to the others through its own shared column and
// barrier.  Look-ahead: the owner of column c+1 applies the update of column
// c to that column first and finishes it before its other updates, so the
// hand-off of every column waits for one update and one pivot only.  (FP64
// instructions take about 64 cycles of an SM sub-partition's FP64 pipe
// each, whatever the active lanes, so the chain's cost is its count of FP64
// instructions, and the trailing updates of two high columns share one
// instruction.)  A warp's registers shift by one column each time it
// finishes one, so its next column is always a[0] and register indices stay
// compile-time constants in a loop over columns that is not unrolled: a long
// unrolled body misses the instruction cache each time the loop jumps back.
// The sequence of operations on every entry (updates in column order, the
// pivot, the scaling) is that of the plain column-by-column algorithm.
// (An LDL' form with four FP64 instructions per pivot instead of six, and a
// schedule that defers each warp's non-urgent updates to just after its own
// pivot, measured 18% fewer cycles per column in its loop but no faster in
// the pipeline: its square roots and scaling after the loop lie on the
// critical path, where this form has only the 1/L_cc of the stored seeds.)
__device__ __forceinline__ void diag_chol_block(double* A, int64_t lda, Dim nd, int64_t k0,
                                                int b, DevState* st, const int64_t* rdev,
                                                uint8_t* accepted, double* dinv, int spd,
                                                DiagScratch& sc) {
  const int64_t n = eval_dim(nd, rdev);
  if (k0 >= n) return;
  const int bw = (int)((n - k0) < b ? (n - k0) : b);
  double(&colbuf)[32][32] = sc.col;
  uint64_t* colbar = sc.bar;
  double* y0_s = sc.y0;
  double* e_s = sc.e;
  int* acc_s = sc.acc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < 32) col_init(&colbar[threadIdx.x], 32);
  bar_sync(3, kDiagThreads);  // the barriers are initialised for all four warps
  // the pivot test d > tol on the bit patterns (tol >= 0: a negative d, -0
  // and NaN compare below or are excluded; +inf passes as it does in FP64)
  const long long tolbits = __double_as_longlong(spd ? 0.0 : st->tol);
  // a[q]: this lane's entry of column jn + 4q, jn = this warp's next column
  // to finish (jn = w + 4 * columns finished)
  int jn = w;
  double a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = w + kDiagWarps * q;
    // L2 loads: other CTAs of a fused launch may have just written the block
    a[q] = (lane < bw && j < bw && j <= lane) ? __ldcg(A + (k0 + lane) * lda + (k0 + j)) : 0.0;
  }
  // The warp's four high columns (>= 16) have entries in rows 16..31 only,
  // so two of them share a register until the low ones are done: pk[h]
  // holds column w + 16 + 8h in lanes 0-15 and column w + 20 + 8h in lanes
  // 16-31, row 16 + (lane & 15); an update instruction then does the work
  // of two (an FP64 instruction costs the same whatever its active lanes).
  const int prow = 16 + (lane & 15);
  double pk[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int jp = w + 16 + 8 * h + (lane < 16 ? 0 : 4);
    pk[h] = (prow < bw && jp < bw && jp <= prow) ? __ldcg(A + (k0 + prow) * lda + (k0 + jp)) : 0.0;
  }
  bool packed = true;
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
    colbuf[c][lane] = l;
    if (lane == c) {
      acc_s[c] = ok;
      y0_s[c] = y0;
      e_s[c] = e;
    }
    return l;
  };
  // column jn is final in a[0]: store it and shift the registers by one
  // column; after the fourth, the high columns go back to lane = row
  auto retire = [&]() {
    if (jn < bw && lane < bw && lane >= jn) A[(k0 + lane) * lda + (k0 + jn)] = a[0];
#pragma unroll
    for (int q = 0; q < 3; ++q) a[q] = a[q + 1];
    a[3] = 0.0;
    jn += kDiagWarps;
    if (packed && jn == w + 16) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const double lo = __shfl_sync(0xffffffffu, pk[h], (lane - 16) & 31);
        a[2 * h] = lane >= 16 ? lo : 0.0;
        a[2 * h + 1] = lane >= 16 ? pk[h] : 0.0;
      }
      packed = false;
    }
  };
  bool timed_out = false;
  if (w == 0) {
    a[0] = pivot(0, a[0]);
    col_publish(&colbar[0]);
    retire();
  }
  // One iteration per column, the same code for every column (a loop body
  // small enough to stay in the instruction cache across iterations).
#pragma unroll 1
  for (int c = 0; c < bw; ++c) {
    if (w != (c & (kDiagWarps - 1))) timed_out |= !col_wait(&colbar[c]);
    else __syncwarp();
    const double li = colbuf[c][lane];
    const int nxt = c + 1;
    if (nxt < bw && w == (nxt & (kDiagWarps - 1))) {
      // this warp owns column c+1 (its a[0]): last update, pivot, hand-off
      if (lane >= nxt) a[0] = fma(-li, colbuf[c][nxt], a[0]);
      a[0] = pivot(nxt, a[0]);
      col_publish(&colbar[nxt]);
      retire();
    }
    // the update of column c on this warp's remaining columns (the same
    // operation on every entry, in the same order, packed or not)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = jn + kDiagWarps * q;
      if (j < bw && lane >= j && (!packed || j < 16)) a[q] = fma(-li, colbuf[c][j], a[q]);
    }
    if (packed) {
      const double lr = colbuf[c][prow];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jp = w + 16 + 8 * h + (lane < 16 ? 0 : 4);
        if (jp < bw && prow < bw && prow >= jp) pk[h] = fma(-lr, colbuf[c][jp], pk[h]);
      }
    }
  }
  if (timed_out && lane == 0) atomicOr(&st->status, ST_TIMEOUT);
  bar_sync(3, kDiagThreads);  // the four warps only (the caller's CTA may be larger)
  if (threadIdx.x < 32) col_inval(&colbar[threadIdx.x]);
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
