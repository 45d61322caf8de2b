// Shared definitions of the cpinv CUDA library (device side and host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cpinv {

// A matrix dimension that may depend on the numerical rank r, which lives in
// device memory (it is decided by the pivot tests on the GPU):
//   value = clamp(off + sel * r, 0, max)
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

__device__ __forceinline__ int64_t eval_dim(const Dim& d, const int64_t* rdev) {
  int64_t v = d.off + (d.sel ? *rdev : 0);
  v = v < 0 ? 0 : v;
  return v > d.max ? d.max : v;
}

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
  int64_t pad[3];
};
static_assert(sizeof(DevState) == 64, "DevState layout");

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
  // batch of nz products (FP64 path): product z uses A + z*zA, B + z*zB,
  // C + z*zC and dimension offsets M.off + z*zM, N.off + z*zN, K.off + z*zK
  int64_t zA, zB, zC;
  int32_t zM, zN, zK, nz;
};

}  // namespace cpinv
