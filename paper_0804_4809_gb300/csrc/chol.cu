// Full-rank Cholesky factorisation with device-side pivot tests (Appendix of
// the paper), blocked by panels of width b <= 32, plus the small kernels
// around it: the pivot tolerance, the column compaction and the diagonal
// blocks of the triangular inverse.
//
// Layout: the factorisation runs in place on the lower triangle of the
// row-major n x n Gram matrix A, in *uncompacted* coordinates: column c of
// the working factor L_full belongs to pivot c, and is entirely zero when
// pivot c is rejected.  Every launch therefore has a host-known shape; the
// kept columns are gathered into the compact n x r factor L afterwards.
//
// Panel p (columns k0 .. k0+bw-1):
//   1. diag kernel: one CTA of four warps factors the bw x bw diagonal block
//      in registers, column by column -- pivot d = A_cc minus the earlier
//      in-block terms; kept iff d > tol (strict, NaN rejected, Appendix);
//      L_cc = sqrt(d) and the column below is divided by it; a rejected
//      column is zeroed.  It records 1/L_cc (0 for a rejected pivot).
//   2. panel kernel: every row below the block solves x T' = a by forward
//      substitution against the block factor T (one warp per row, many
//      CTAs), so L_full(below, panel) needs no explicit block inverse.
//   3. trailing update A(trailing) -= L_full(trailing, panel) L_full(..)'
//      (right-looking FP64 form) or, in the exact-slice form, the next
//      panel's left-looking update from residue planes (chol_exact.cu).
#include <cmath>

#include "chol_device.cuh"
#include "common.cuh"
#include "kernels.h"

namespace cpinv {

namespace {

// tol = rel_tol * min{A_jj : A_jj > 0}; flags non-finite diagonal entries
// (a NaN or Inf anywhere in G reaches the diagonal of its Gram column/row).
__global__ void tol_kernel(const double* A, int64_t lda, int64_t n, double rel_tol,
                           DevState* st) {
  __shared__ double smin[256];
  __shared__ int sbad[256];
  double mn = INFINITY;
  int bad = 0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double d = A[j * lda + j];
    if (!isfinite(d)) bad = 1;
    else if (d > 0.0 && d < mn) mn = d;
  }
  smin[threadIdx.x] = mn;
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      sbad[threadIdx.x] |= sbad[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = smin[0];
    const int has = m < INFINITY;
    st->has_pos = has;
    st->min_pos = has ? m : 0.0;
    // With no positive diagonal entry every pivot test must fail.
    st->tol = has ? rel_tol * m : INFINITY;
    if (sbad[0]) atomicOr(&st->status, ST_NONFINITE);
  }
}

__global__ void __launch_bounds__(chol::kDiagThreads) diag_chol_kernel(double* A, int64_t lda, Dim nd,
                                                                 int64_t k0, int b, DevState* st,
                                                                 const int64_t* rdev,
                                                                 uint8_t* accepted, double* dinv,
                                                                 int spd) {
  __shared__ chol::DiagScratch sc;
  chol::diag_chol_block(A, lda, nd, k0, b, st, rdev, accepted, dinv, spd, sc);
}

// One block per problem of a batch of equal-shaped problems (strides in
// elements; st and the rank are per problem).
__global__ void __launch_bounds__(chol::kDiagThreads) diag_chol_batched_kernel(DiagBatch p) {
  const int64_t z = blockIdx.x;
  DevState* st = p.st + z;
  __shared__ chol::DiagScratch sc;
  chol::diag_chol_block(p.A + z * p.zA, p.lda, p.nd, p.k0, p.b, st, &st->rank,
                        p.accepted ? p.accepted + z * p.zAcc : nullptr, p.dinv + z * p.zDinv,
                        p.spd, sc);
}

// Rows below the diagonal block of panel k0: L(i, P) solves L(i, P) T' =
// A(i, P) by forward substitution, T = the factored block (rejected
// columns zero, 1/T_cc = dinv[c], 0 when rejected).  One warp per row, lane
// c for column c; in place.
constexpr int kPanelRows = 8;

__device__ __forceinline__ void panel_solve_rows(double* A, int64_t lda, Dim nd,
                                                 const int64_t* rdev, int64_t k0, int b,
                                                 const double* dinv) {
  const int64_t n = eval_dim(nd, rdev);
  if (k0 >= n) return;
  const int bw = (int)((n - k0) < b ? (n - k0) : b);
  // Ts[r][c] = T(r, c) / T(c, c): the substitution chain is then one shuffle
  // and one fused multiply-add per column, x_c = acc_c / T(c, c) at the end
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
  const int64_t i = k0 + bw + (int64_t)blockIdx.x * kPanelRows + (threadIdx.x >> 5);
  if (i >= n) return;
  double acc = lane < bw ? A[i * lda + k0 + lane] : 0.0;
  for (int c = 0; c < bw; ++c) {
    const double ac = __shfl_sync(0xffffffffu, acc, c);
    if (lane > c) acc = fma(-ac, Ts[lane][c], acc);
  }
  if (lane < bw) A[i * lda + k0 + lane] = acc * dv[lane];
}

__global__ void __launch_bounds__(32 * kPanelRows) panel_solve_kernel(double* A, int64_t lda,
                                                                      Dim nd, const int64_t* rdev,
                                                                      int64_t k0, int b,
                                                                      const double* dinv) {
  panel_solve_rows(A, lda, nd, rdev, k0, b, dinv);
}

__global__ void __launch_bounds__(32 * kPanelRows) panel_solve_batched_kernel(PanelBatch p) {
  const int64_t z = blockIdx.y;
  panel_solve_rows(p.A + z * p.zA, p.lda, p.nd, &p.st[z].rank, p.k0, p.b, p.dinv + z * p.zDinv);
}

// Inverse of each b x b diagonal block of the lower-triangular T (order r):
// Tinv[q] (row-major b x b, zero past r).  One CTA of 32 warps per block,
// grid.y over a batch; warp j solves T_qq w = e_j by forward substitution.
__global__ void __launch_bounds__(1024) tri_block_inverse_kernel(const double* T, int64_t ld,
                                                                 int64_t zT, const int64_t* rdev,
                                                                 int64_t zR, int b, double* Tinv,
                                                                 int64_t zTinv) {
  const int64_t z = blockIdx.y;
  T += z * zT;
  Tinv += z * zTinv;
  const int64_t r = rdev[z * zR];
  const int64_t k0 = (int64_t)blockIdx.x * b;
  double* out = Tinv + (int64_t)blockIdx.x * b * b;
  const int i = threadIdx.x & 31, j = threadIdx.x >> 5;
  if (k0 >= r) {
    if (i < b && j < b) out[i * b + j] = 0.0;
    return;
  }
  const int bw = (int)((r - k0) < b ? (r - k0) : b);
  __shared__ double Ts[32][33];
  __shared__ double rinv[32];
  Ts[i][j] = (i < bw && j < bw && j <= i) ? T[(k0 + i) * ld + (k0 + j)] : 0.0;
  __syncthreads();
  // 1/T_kk for every k by one warp (an FP64 division is a long run of FP64
  // instructions, each costing the same with one active lane as with 32)
  if (j == 0) rinv[i] = i < bw ? 1.0 / Ts[i][i] : 0.0;
  __syncthreads();
  double w = 0.0;
  if (j < bw) {
    // w_k = (delta_kj - sum_{l<k} T_kl w_l) / T_kk for k = j..bw-1
    double x = 0.0;
    for (int k = j; k < bw; ++k) {
      double v = 0.0;
      if (i == k) v = ((k == j ? 1.0 : 0.0) - x) * rinv[k];
      const double wk = __shfl_sync(0xffffffffu, v, k);
      if (i == k) w = wk;
      if (i > k) x = fma(Ts[i][k], wk, x);
    }
  }
  if (i < b && j < b) out[i * b + j] = (i < bw && j < bw && i >= j) ? w : 0.0;
}

// Prefix sum of the kept-pivot mask: colidx[c] = index of pivot c among the
// kept ones (or -1), and the rank r.  One CTA.
__global__ void scan_kernel(const uint8_t* accepted, int64_t n, int32_t* colidx, DevState* st) {
  __shared__ int32_t part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t chunk = (n + nt - 1) / nt;
  const int64_t beg = tid * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  int32_t cnt = 0;
  for (int64_t c = beg; c < end; ++c) cnt += accepted[c] ? 1 : 0;
  part[tid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int32_t run = 0;
    for (int t = 0; t < nt; ++t) {
      const int32_t v = part[t];
      part[t] = run;
      run += v;
    }
    st->rank = run;
  }
  __syncthreads();
  int32_t run = part[tid];
  for (int64_t c = beg; c < end; ++c) {
    if (accepted[c]) colidx[c] = run++;
    else colidx[c] = -1;
  }
}

// L(i, colidx[c]) = L_full(i, c) for kept c (0 above the diagonal).
__global__ void gather_kernel(const double* Lfull, int64_t lda, int64_t n, const int32_t* colidx,
                              double* L, int64_t ldl) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, c = e % n;
    const int32_t j = colidx[c];
    if (j >= 0) L[i * ldl + j] = (c <= i) ? Lfull[i * lda + c] : 0.0;
  }
}

// Diagonal blocks of W = U^-1 from the stored block inverses, and zeros
// elsewhere in the r x r leading part (row-major, ld = ldw).
__global__ void tri_inv_init_kernel(double* W, int64_t ldw, int64_t nmax, const int64_t* rdev,
                                    const double* Tinv, int b) {
  const int64_t r = *rdev;
  const int64_t total = nmax * nmax;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nmax, j = e % nmax;
    double v = 0.0;
    if (i < r && j < r && i / b == j / b && j <= i) {
      const int64_t p = i / b;
      v = Tinv[p * (int64_t)b * b + (i - p * b) * b + (j - p * b)];
    }
    W[i * ldw + j] = v;
  }
}

// Copy the lower triangle onto the upper one (C symmetric, order from rdev or host).
__global__ void mirror_kernel(double* C, int64_t ldc, Dim nd, const int64_t* rdev) {
  const int64_t n = eval_dim(nd, rdev);
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (j > i) C[i * ldc + j] = C[j * ldc + i];
  }
}

__global__ void copy_mask_kernel(const uint8_t* src, uint8_t* dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

inline unsigned grid_for(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_tol(const double* A, int64_t lda, int64_t n, double rel_tol, DevState* st,
                       cudaStream_t s) {
  tol_kernel<<<1, 256, 0, s>>>(A, lda, n, rel_tol, st);
  return cudaGetLastError();
}

cudaError_t launch_diag_factor(double* A, int64_t lda, Dim nd, int64_t k0, int b, DevState* st,
                               const int64_t* rdev, uint8_t* accepted, double* dinv, int spd,
                               cudaStream_t s) {
  if (b > 32 || b < 1) return cudaErrorInvalidValue;
  diag_chol_kernel<<<1, chol::kDiagThreads, 0, s>>>(A, lda, nd, k0, b, st, rdev, accepted, dinv, spd);
  return cudaGetLastError();
}

cudaError_t launch_diag_batched(const DiagBatch& p, int nz, cudaStream_t s) {
  if (p.b > 32 || p.b < 1) return cudaErrorInvalidValue;
  if (nz <= 0) return cudaSuccess;
  diag_chol_batched_kernel<<<nz, chol::kDiagThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_panel_solve(double* A, int64_t lda, Dim nd, const int64_t* rdev, int64_t k0,
                               int b, const double* dinv, cudaStream_t s) {
  if (b > 32 || b < 1) return cudaErrorInvalidValue;
  const int64_t rows = nd.max - k0 - b;
  if (rows <= 0) return cudaSuccess;
  panel_solve_kernel<<<(unsigned)((rows + kPanelRows - 1) / kPanelRows), 32 * kPanelRows, 0, s>>>(
      A, lda, nd, rdev, k0, b, dinv);
  return cudaGetLastError();
}

cudaError_t launch_panel_solve_batched(const PanelBatch& p, int nz, cudaStream_t s) {
  if (p.b > 32 || p.b < 1) return cudaErrorInvalidValue;
  const int64_t rows = p.nd.max - p.k0 - p.b;
  if (rows <= 0 || nz <= 0) return cudaSuccess;
  if (nz > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)((rows + kPanelRows - 1) / kPanelRows), (unsigned)nz);
  panel_solve_batched_kernel<<<grid, 32 * kPanelRows, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tri_block_inverse(const double* T, int64_t ld, int64_t nmax,
                                     const int64_t* rdev, int b, double* Tinv, cudaStream_t s) {
  return launch_tri_block_inverse_batched(T, ld, 0, nmax, rdev, 0, b, Tinv, 0, 1, s);
}

cudaError_t launch_tri_block_inverse_batched(const double* T, int64_t ld, int64_t zT,
                                             int64_t nmax, const int64_t* rdev, int64_t zR, int b,
                                             double* Tinv, int64_t zTinv, int nz,
                                             cudaStream_t s) {
  if (b < 1 || b > 32) return cudaErrorInvalidValue;
  if (nmax <= 0 || nz <= 0) return cudaSuccess;
  if (nz > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)((nmax + b - 1) / b), (unsigned)nz);
  tri_block_inverse_kernel<<<grid, 1024, 0, s>>>(T, ld, zT, rdev, zR, b, Tinv, zTinv);
  return cudaGetLastError();
}

cudaError_t launch_scan(const uint8_t* accepted, int64_t n, int32_t* colidx, DevState* st,
                        cudaStream_t s) {
  scan_kernel<<<1, 1024, 0, s>>>(accepted, n, colidx, st);
  return cudaGetLastError();
}

cudaError_t launch_gather(const double* Lfull, int64_t lda, int64_t n, const int32_t* colidx,
                          double* L, int64_t ldl, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_kernel<<<grid_for(n * n, 256), 256, 0, s>>>(Lfull, lda, n, colidx, L, ldl);
  return cudaGetLastError();
}

cudaError_t launch_tri_inv_init(double* W, int64_t ldw, int64_t nmax, const int64_t* rdev,
                                const double* Tinv, int b, cudaStream_t s) {
  if (nmax <= 0) return cudaSuccess;
  tri_inv_init_kernel<<<grid_for(nmax * nmax, 256), 256, 0, s>>>(W, ldw, nmax, rdev, Tinv, b);
  return cudaGetLastError();
}

cudaError_t launch_mirror(double* C, int64_t ldc, Dim nd, const int64_t* rdev, cudaStream_t s) {
  if (nd.max <= 0) return cudaSuccess;
  mirror_kernel<<<grid_for(nd.max * nd.max, 256), 256, 0, s>>>(C, ldc, nd, rdev);
  return cudaGetLastError();
}

cudaError_t launch_copy_mask(const uint8_t* src, uint8_t* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  copy_mask_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace cpinv
