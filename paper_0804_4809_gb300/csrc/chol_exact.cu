// Left-looking full-rank Cholesky whose panel updates are exact residue
// products on the tensor cores (exact-slice mode; Appendix of the paper).
//
// Every row of the factor is bounded by its diagonal entry: the kept and the
// rejected parts of row i together sum to A_ii, so |L_ij| <= sqrt(A_ii).  That
// bound fixes a power-of-two scale per row before any column exists, so each
// finished panel of L is cut into residues once, into a persistent set of
// residue planes RL[j][row][col]; the update of panel p,
//   A(k0:n, P) -= L(k0:n, 0:k0) L(P, 0:k0)',
// is then one tensor-core product over those planes (no re-splitting) and
// one CRT reconstruction that subtracts the exactly summed update from A.
#include <cmath>

#include "common.cuh"
#include "crt.h"
#include "crt_device.cuh"
#include "kernels.h"

namespace cpinv {
namespace {

// E[i] = biased exponent of sqrt(A_ii), plus one: |L_ij| < 2^(E[i] - 1022).
// 0 for a non-positive or non-finite diagonal entry (that row of L is 0).
__global__ void rowscale_kernel(const double* A, int64_t lda, Dim nd, const int64_t* rdev,
                                int64_t rows_max, int32_t* E) {
  const int64_t n = eval_dim(nd, rdev);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows_max;
       i += (int64_t)gridDim.x * blockDim.x) {
    int e = 0;
    if (i < n) {
      const double d = A[i * lda + i];
      if (d > 0.0 && isfinite(d)) {
        const uint64_t b = (uint64_t)__double_as_longlong(sqrt(d));
        e = (int)((b >> 52) & 0x7FF) + 1;
      }
    }
    E[i] = e;
  }
}

// Rows [k0, n) of panel k0: below the diagonal block, L(i, P) solves
// L(i, P) T' = A(i, P) by forward substitution against the factored block T
// (1/T_cc = dinv[c], 0 for a rejected pivot; in place); every row of the
// panel (diagonal block included) is then cut into residues with the row
// scale E[i] and written to RL[j][i][k0 + c].  One warp per row, lane c for
// column c; many CTAs (the FP64 pipe of each SM is narrow).
constexpr int kPanelRows = 8;

__global__ void __launch_bounds__(256) panel_solve_split_kernel(
    double* A, int64_t lda, Dim nd, const int64_t* rdev, int64_t k0, int b, const double* dinv,
    const int32_t* E, int n_mod, int beta, __nv_bfloat16* RL, int64_t rl_rows, int64_t rl_kpad) {
  const int64_t n = eval_dim(nd, rdev);
  if (k0 >= n) return;
  const int bw = (int)((n - k0) < b ? (n - k0) : b);
  // Ts[r][c] = T(r, c) / T(c, c) below the diagonal (see panel_solve_rows)
  __shared__ double Ts[32][33];
  __shared__ double dv[32];
  if (threadIdx.x < 32) dv[threadIdx.x] = threadIdx.x < bw ? dinv[threadIdx.x] : 0.0;
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    Ts[r][c] = (r < bw && c < r) ? A[(k0 + r) * lda + (k0 + c)] * dv[c] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t i = k0 + (int64_t)blockIdx.x * kPanelRows + (threadIdx.x >> 5);
  if (i >= n) return;
  double l = 0.0;
  if (i >= k0 + bw) {
    double acc = lane < bw ? A[i * lda + k0 + lane] : 0.0;
    for (int c = 0; c < bw; ++c) {
      const double ac = __shfl_sync(0xffffffffu, acc, c);
      if (lane > c) acc = fma(-ac, Ts[lane][c], acc);
    }
    l = acc * dv[lane];
    if (lane < bw) A[i * lda + k0 + lane] = l;
  } else if (lane < bw && lane <= i - k0) {
    l = A[i * lda + k0 + lane];  // diagonal block: already the factor
  }
  if (lane < bw) {
    const uint64_t bits = (uint64_t)__double_as_longlong(l);
    const uint64_t a = crt::integerize(bits, E[i], beta);
    crt::store_residues(a, (bits >> 63) != 0, n_mod, RL + (size_t)i * rl_kpad + (k0 + lane),
                        (size_t)rl_rows * (size_t)rl_kpad);
  }
}

inline unsigned grid1d(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 8) g = 152 * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_rowscale(const double* A, int64_t lda, Dim nd, const int64_t* rdev,
                            int64_t rows_max, int32_t* E, cudaStream_t s) {
  rowscale_kernel<<<grid1d(rows_max, 256), 256, 0, s>>>(A, lda, nd, rdev, rows_max, E);
  return cudaGetLastError();
}

cudaError_t launch_panel_solve_split(double* A, int64_t lda, Dim nd, const int64_t* rdev,
                                     int64_t k0, int b, const double* dinv, const int32_t* E,
                                     int n_mod, int beta, void* RL, int64_t rl_rows,
                                     int64_t rl_kpad, cudaStream_t s) {
  if (b > 32) return cudaErrorInvalidValue;
  const int64_t rows = nd.max - k0;
  if (rows <= 0) return cudaSuccess;
  panel_solve_split_kernel<<<(unsigned)((rows + kPanelRows - 1) / kPanelRows), 256, 0, s>>>(
      A, lda, nd, rdev, k0, b, dinv, E, n_mod, beta, (__nv_bfloat16*)RL, rl_rows, rl_kpad);
  return cudaGetLastError();
}

}  // namespace cpinv
