// Shared definitions of the cpinv CUDA library (device side and host side).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace cpinv {

// A matrix dimension that may depend on a value that lives in device memory,
// such as the numerical rank r (it is decided by the pivot tests on the GPU):
//   value = clamp(off + v, 0, max),  v = rdev[sel - 1] for sel > 0,
//                                    v = -rdev[-sel - 1] for sel < 0, 0 for sel = 0
// where rdev points at a DevState (sel = 1: the rank; SEL_M / SEL_N: the
// problem's own m and n in a batch; sel = -1: minus the rank, e.g. n - r).
// With sel = 0 it is the plain host value `off` (max >= off).
struct Dim {
  int64_t off;
  int64_t max;
  int32_t sel;
  int32_t pad;
};

__host__ __device__ inline Dim hdim(int64_t v) { return Dim{v, v, 0, 0}; }
// r + off, clamped to [0, max]
__host__ __device__ inline Dim rdim(int64_t off, int64_t max) { return Dim{off, max, 1, 0}; }
// off - r, clamped to [0, max]
__host__ __device__ inline Dim ddim(int64_t off, int64_t max) { return Dim{off, max, -1, 0}; }

__device__ __forceinline__ int64_t eval_dim(const Dim& d, const int64_t* rdev) {
  int64_t v = d.off + (d.sel > 0 ? rdev[d.sel - 1] : d.sel < 0 ? -rdev[-d.sel - 1] : 0);
  v = v < 0 ? 0 : v;
  return v > d.max ? d.max : v;
}

// Inner index of a nested batch z = zo nzi + zi (zo: a problem, zi: a block
// inside it): the inner blocks' operand stride and the offset added per inner
// block to their dims.
struct ZNest {
  int32_t nzi;
  int64_t zXi, zoff;
};

// Status bits recorded by kernels (OR-ed into DevState::status).
enum : int32_t { ST_NONFINITE = 1, ST_NUMERICAL = 2, ST_TIMEOUT = 4 };

// Per-call device state, at the start of the workspace.
struct DevState {
  int64_t rank;     // numerical rank r of the Gram factorisation
  int64_t rank_n;   // kept pivots when factoring N = L'L (must equal rank)
  int32_t status;   // ST_* bits
  int32_t has_pos;  // 1 if some diagonal entry of A is > 0
  double tol;       // Appendix: rel_tol * min positive diagonal entry
  double min_pos;   // that minimum
  int64_t dim_m;    // batched problems: this problem's m and n (else 0)
  int64_t dim_n;
  int64_t panel_flag;  // block-row CTAs done (exact factorisation, cumulative over launches)
  int64_t diag_count;  // diagonal-block update CTAs done (exact factorisation, cumulative)
  int64_t spare[7];
};
static_assert(sizeof(DevState) == 128, "DevState layout");
// Dim::sel values that read DevState::dim_m and DevState::dim_n
enum : int32_t { SEL_RANK = 1, SEL_M = 6, SEL_N = 7 };
static_assert(offsetof(DevState, dim_m) == 8 * (SEL_M - 1), "SEL_M");
static_assert(offsetof(DevState, dim_n) == 8 * (SEL_N - 1), "SEL_N");
__host__ __device__ inline Dim mdim(int64_t max) { return Dim{0, max, SEL_M, 0}; }
__host__ __device__ inline Dim ndim(int64_t off, int64_t max) { return Dim{off, max, SEL_N, 0}; }

// Row-major matrix operand of a product C = alpha * op(A) op(B) + beta * C.
// Element (i, k) of op(A) is  A[i*ld + k]  when !trans, else A[k*ld + i].
struct GemmParams {
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  Dim M, N, K;
  double alpha, beta;
  const int64_t* rdev;  // device rank, read when a Dim has sel = 1
  int32_t lower;        // 1: only C(i, j) with i >= j is computed and written
  int32_t pad;          // FP64 path: 1 if C aliases A or B (whole-row tiles)
  // batch of nz products (FP64 path).  Index z = zi + nzi * zo when nzi > 1
  // (two levels, e.g. the nodes of a level x the problems of a batch), else
  // zi = z, zo = 0.  Product z uses A + zi*zA + zo*oA (B, C alike), rdev +
  // zi*zR + zo*oR and dimension offsets M.off + zi*zM, N.off + zi*zN,
  // K.off + zi*zK.
  int64_t zA, zB, zC;
  int32_t zM, zN, zK, nz;
  int64_t zR;
  int64_t oA, oB, oC, oR;
  int32_t nzi;
  int32_t pad2;
};

}  // namespace cpinv
