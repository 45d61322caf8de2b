// Full-rank Cholesky factorisation with device-side pivot tests (Appendix of
// the paper), blocked by panels of width b <= 64, plus the small kernels
// around it: the pivot tolerance, the column compaction and the diagonal
// blocks of the triangular inverse.
//
// Layout: the factorisation runs in place on the lower triangle of the
// row-major n x n Gram matrix A, in *uncompacted* coordinates: column c of
// the working factor L_full belongs to pivot c, and is entirely zero when
// pivot c is rejected.  Every launch therefore has a host-known shape; the
// kept columns are gathered into the compact n x r factor L afterwards.
//
// Panel p (columns k0 .. k0+bw-1), right-looking:
//   1. diag_factor_kernel: one CTA factors the bw x bw diagonal block in
//      shared memory column by column -- pivot d = A_cc minus the earlier
//      in-block terms; kept iff d > tol (strict, NaN rejected, Appendix);
//      L_cc = sqrt(d) and the column below is divided by it; a rejected
//      column is zeroed.  It then forms Z, the bw x bw matrix with
//      L_full(below, panel) = A(below, panel) Z, i.e. Z = (T^-1)' on the kept
//      rows/columns (T = the kept rows and columns of the block factor) and 0
//      elsewhere, so the panel below the block is one matrix product.
//   2. A(below, panel) := A(below, panel) Z          (product, in place)
//   3. A(trailing) -= L_full(trailing, panel) L_full(trailing, panel)'  (lower)
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace cpinv {

namespace {

constexpr int MAXB = 64;

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

// One CTA factors the diagonal block of panel `k0` (see the file comment).
// `nd` is the order of the matrix being factored (host value, or the device
// rank when factoring N = L'L).  spd = 1: tolerance 0 and every pivot must be
// kept (else ST_NUMERICAL); the block inverse T^-1 is stored in Tinv.
__global__ void __launch_bounds__(256) diag_factor_kernel(double* A, int64_t lda, Dim nd,
                                                          int64_t k0, int b, DevState* st,
                                                          const int64_t* rdev, uint8_t* accepted,
                                                          double* Z, double* Tinv, int spd) {
  const int64_t n = eval_dim(nd, rdev);
  if (k0 >= n) return;
  const int bw = (int)((n - k0) < b ? (n - k0) : b);
  // dynamic shared memory: S and Wi (b x (b+1) doubles each), then acc (b ints)
  extern __shared__ double smem[];
  const int ls = b + 1;
  double* Sm = smem;
  double* Wm = smem + b * ls;
  int* acc = (int*)(smem + 2 * b * ls);
#define S(i, j) Sm[(i) * ls + (j)]
#define Wi(i, j) Wm[(i) * ls + (j)]
  const int tid = threadIdx.x, nt = blockDim.x;
  const double tol = spd ? 0.0 : st->tol;

  for (int e = tid; e < bw * bw; e += nt) {
    const int i = e / bw, j = e % bw;
    S(i, j) = (j <= i) ? A[(k0 + i) * lda + (k0 + j)] : 0.0;
  }
  __syncthreads();

  for (int c = 0; c < bw; ++c) {
    const double d = S(c, c);
    const bool ok = d > tol;  // false for NaN
    __syncthreads();
    if (ok) {
      const double piv = sqrt(d);
      for (int i = c + 1 + tid; i < bw; i += nt) S(i, c) /= piv;
      if (tid == 0) S(c, c) = piv;
      __syncthreads();
      const int rem = bw - c - 1;
      for (int e = tid; e < rem * rem; e += nt) {
        const int ii = e / rem, jj = e % rem;
        if (jj <= ii) S(c + 1 + ii, c + 1 + jj) -= S(c + 1 + ii, c) * S(c + 1 + jj, c);
      }
    } else {
      for (int i = c + tid; i < bw; i += nt) S(i, c) = 0.0;
    }
    if (tid == 0) acc[c] = ok ? 1 : 0;
    __syncthreads();
  }

  // Inverse of T' := the block factor with every rejected row replaced by the
  // identity row; on the kept rows/columns it equals T^-1.  Column j by thread j.
  if (tid < bw) {
    const int j = tid;
    for (int i = 0; i < j; ++i) Wi(i, j) = 0.0;
    const double djj = acc[j] ? S(j, j) : 1.0;
    Wi(j, j) = 1.0 / djj;
    for (int i = j + 1; i < bw; ++i) {
      double v;
      if (acc[i]) {
        double s = 0.0;
        for (int k = j; k < i; ++k) s = fma(S(i, k), Wi(k, j), s);
        v = -s / S(i, i);
      } else {
        v = 0.0;
      }
      Wi(i, j) = v;
    }
  }
  __syncthreads();

  // Write back the block of L_full (lower part), Z, the mask and T^-1.
  for (int e = tid; e < bw * bw; e += nt) {
    const int i = e / bw, j = e % bw;
    if (j <= i) A[(k0 + i) * lda + (k0 + j)] = S(i, j);
    // Z(c, j) = (T^-1)(j, c) on kept c and j, else 0.
    const int c = i;
    Z[c * b + j] = (acc[c] && acc[j]) ? Wi(j, c) : 0.0;
    if (spd && Tinv) Tinv[i * b + j] = Wi(i, j);
  }
  if (tid == 0) {
    int kept = 0;
    for (int c = 0; c < bw; ++c) kept += acc[c];
    if (spd) {
      if (kept != bw) atomicOr(&st->status, ST_NUMERICAL);
      atomicAdd((unsigned long long*)&st->rank_n, (unsigned long long)kept);
    }
  }
  if (!spd && accepted)
    for (int c = tid; c < bw; c += nt) accepted[k0 + c] = (uint8_t)acc[c];
}
#undef S
#undef Wi

// 1/sqrt(d) for d > 0 by Newton's iteration y <- y (3 - d y^2) / 2 from a
// single-precision seed (about 22 correct bits); two FP64 steps bring it to
// full double precision (each step doubles the correct bits).  Ranges beyond
// float are handled by scaling d with an even power of two.
__device__ __forceinline__ double rsqrt_newton(double d) {
  int e2 = 0;
  double ds = d;
  if (d > 1e36 || d < 1e-36) {
    e2 = (ilogb(d) / 2) * 2;
    ds = scalbn(d, -e2);
  }
  double y = (double)rsqrtf((float)ds);
  const double h = 0.5 * ds;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return e2 ? scalbn(y, -e2 / 2) : y;
}

// The same factorisation for b <= 32, one warp per column of the block and
// one lane per row: thread (lane i, warp j) keeps A(i, j) in a register.  The
// FP64 pipe of one SM is narrow, so the mapping keeps the FP64 instructions
// per pivot to a minimum: the pivot (one lane), the column scaling (one warp
// instruction), and one fused multiply-add per trailing column warp; two
// barriers per column.  The inverse of the identity-patched block factor is
// then 32 independent forward substitutions, warp j solving T w = e_j with
// shuffles only.
__device__ __forceinline__ void diag32_block(double* A, int64_t lda, Dim nd, int64_t k0, int b,
                                             DevState* st, const int64_t* rdev, uint8_t* accepted,
                                             double* Z, double* Tinv, int spd) {
  const int64_t n = eval_dim(nd, rdev);
  if (k0 >= n) return;
  const int bw = (int)((n - k0) < b ? (n - k0) : b);
  __shared__ double Ls[32][33];   // Ls[row][col] = L(row, col)
  __shared__ double colc[32];
  __shared__ double dinv[32];
  __shared__ int acc[32];
  __shared__ int ok_s;
  const int i = threadIdx.x & 31;   // row (lane)
  const int j = threadIdx.x >> 5;   // column (warp)
  const bool in = i < bw && j < bw && j <= i;
  const double tol = spd ? 0.0 : st->tol;
  double a = in ? A[(k0 + i) * lda + (k0 + j)] : 0.0;

  for (int c = 0; c < bw; ++c) {
    if (j == c) {
      // warp c: pivot in lane c, then the column
      const double d = __shfl_sync(0xffffffffu, a, c);
      const bool ok = d > tol;  // false for NaN
      double y = 0.0;
      if (ok) y = rsqrt_newton(d);
      if (i == c) {
        a = ok ? d * y : 0.0;   // sqrt(d)
        ok_s = ok ? 1 : 0;
        acc[c] = ok ? 1 : 0;
        dinv[c] = ok ? y : 1.0;  // 1 / L_cc (1 on a rejected row: identity patch)
      } else if (i > c) {
        a = ok ? a * y : 0.0;
      }
      colc[i] = (i >= c) ? a : 0.0;
    }
    __syncthreads();
    if (ok_s && j > c && i >= j && i < bw) a = fma(-colc[i], colc[j], a);
    __syncthreads();
  }
  // a = L(i, j) for j <= i (rejected columns zero).  The inverse below works
  // on T~(i, k) = T(i, k) / T(k, k) of the patched factor T (rejected rows
  // are identity rows): with r the running right-hand side, r_i -= T~(i, k) r_k
  // once r_k is final, and W(i, j) = r_i / T(i, i) at the end.
  Ls[i][j] = (in && acc[i]) ? a * dinv[j] : 0.0;
  __syncthreads();

  // warp j: column j of W = inverse of the patched factor, by forward
  // substitution with shuffles only; lane i ends with W(i, j).
  double w = 0.0;
  if (j < bw) {
    double r = (i == j) ? 1.0 : 0.0;
    for (int k = j; k < bw; ++k) {
      const double rk = __shfl_sync(0xffffffffu, r, k);
      if (i > k) r = fma(-Ls[i][k], rk, r);
    }
    if (i >= j && i < bw) w = r * dinv[i];
  }
  if (i < bw && j < bw) {
    if (j <= i) A[(k0 + i) * lda + (k0 + j)] = a;
    // Z(c, jj) = W(jj, c) on kept c and jj: this thread's W(i, j) is Z(j, i)
    Z[j * b + i] = (acc[i] && acc[j]) ? w : 0.0;
    if (spd && Tinv) Tinv[i * b + j] = w;
  }
  if (threadIdx.x == 0) {
    int kept = 0;
    for (int c = 0; c < bw; ++c) kept += acc[c];
    if (spd) {
      if (kept != bw) atomicOr(&st->status, ST_NUMERICAL);
      atomicAdd((unsigned long long*)&st->rank_n, (unsigned long long)kept);
    }
  }
  if (!spd && accepted && threadIdx.x < bw) accepted[k0 + threadIdx.x] = (uint8_t)acc[threadIdx.x];
}

__global__ void __launch_bounds__(1024) diag32_kernel(double* A, int64_t lda, Dim nd, int64_t k0,
                                                      int b, DevState* st, const int64_t* rdev,
                                                      uint8_t* accepted, double* Z, double* Tinv,
                                                      int spd) {
  diag32_block(A, lda, nd, k0, b, st, rdev, accepted, Z, Tinv, spd);
}

// One block per problem of a batch of equal-shaped problems (strides in
// elements; st and the rank are per problem).
__global__ void __launch_bounds__(1024) diag32_batched_kernel(DiagBatch p) {
  const int64_t z = blockIdx.x;
  DevState* st = p.st + z;
  diag32_block(p.A + z * p.zA, p.lda, p.nd, p.k0, p.b, st, &st->rank,
               p.accepted ? p.accepted + z * p.zAcc : nullptr, p.Z + z * p.zZ,
               p.Tinv ? p.Tinv + z * p.zT : nullptr, p.spd);
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
                               const int64_t* rdev, uint8_t* accepted, double* Z, double* Tinv,
                               int spd, cudaStream_t s) {
  if (b > MAXB || b < 1) return cudaErrorInvalidValue;
  if (b <= 32) {
    diag32_kernel<<<1, 1024, 0, s>>>(A, lda, nd, k0, b, st, rdev, accepted, Z, Tinv, spd);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(double) * 2 * b * (b + 1) + sizeof(int) * b;
  static bool attr_set = false;
  if (!attr_set) {
    const size_t maxsmem = sizeof(double) * 2 * MAXB * (MAXB + 1) + sizeof(int) * MAXB;
    cudaError_t e = cudaFuncSetAttribute(diag_factor_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxsmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  diag_factor_kernel<<<1, 256, smem, s>>>(A, lda, nd, k0, b, st, rdev, accepted, Z, Tinv, spd);
  return cudaGetLastError();
}

cudaError_t launch_diag_batched(const DiagBatch& p, int nz, cudaStream_t s) {
  if (p.b > 32 || p.b < 1) return cudaErrorInvalidValue;
  if (nz <= 0) return cudaSuccess;
  diag32_batched_kernel<<<nz, 1024, 0, s>>>(p);
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
