// Small kernels of the reverse pass of W = G+ F (cpinv_lstsq_backward): the
// bookkeeping of the kept-pivot set S (index lists, the factor's structural
// pattern), row gathers, Phi (lower triangle with the diagonal halved) and the symmetrised
// scatter of the Gram adjoint.  The dense products of the pass go through the
// library's FP64 / exact-slice / split products.
#include "common.cuh"
#include "kernels.h"

namespace cpinv {
namespace {

inline unsigned grid_n(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 8) g = 152 * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

// One CTA: pref[i] = number of kept pivots among 0..i, sidx[c] = the c-th
// kept pivot, didx[j] = the j-th rejected pivot (natural order).
__global__ void __launch_bounds__(1024) pivot_lists_kernel(const uint8_t* acc, int64_t n,
                                                           int32_t* pref, int32_t* sidx,
                                                           int32_t* didx) {
  __shared__ int32_t part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t chunk = (n + nt - 1) / nt;
  const int64_t beg = tid * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  int32_t cnt = 0;
  for (int64_t i = beg; i < end; ++i) cnt += acc[i] ? 1 : 0;
  part[tid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int32_t run = 0;
    for (int t = 0; t < nt; ++t) {
      const int32_t v = part[t];
      part[t] = run;
      run += v;
    }
  }
  __syncthreads();
  int32_t run = part[tid];
  for (int64_t i = beg; i < end; ++i) {
    if (acc[i]) {
      sidx[run] = (int32_t)i;
      ++run;
    } else {
      didx[i - run] = (int32_t)i;
    }
    pref[i] = run;
  }
}

// Lbar(i, c) = 0 where the factor has a structural zero: kept pivot c lies
// after row i (c >= pref[i]).  Columns c < r of an n x r block (ld).
__global__ void pattern_mask_kernel(double* Lb, int64_t ld, int64_t n, const int32_t* pref,
                                    const int64_t* rdev) {
  const int64_t r = *rdev;
  const int64_t total = n * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r, c = e % r;
    if (c >= pref[i]) Lb[i * ld + c] = 0.0;
  }
}

// dst(j, c) = src(idx[j], c) for j < rows (rows = r, or n - r when
// count_rejected), c < r.
__global__ void gather_rows_kernel(const double* src, int64_t lds, const int32_t* idx,
                                   int64_t n, int count_rejected, const int64_t* rdev,
                                   double* dst, int64_t ldd) {
  const int64_t r = *rdev;
  const int64_t rows = count_rejected ? n - r : r;
  const int64_t total = rows * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / r, c = e % r;
    dst[j * ldd + c] = src[(int64_t)idx[j] * lds + c];
  }
}

// P = Phi(P): lower triangle with the diagonal halved, upper part zero
// (order r).
__global__ void phi_kernel(double* P, int64_t ld, const int64_t* rdev) {
  const int64_t r = *rdev;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r, j = e % r;
    double* p = P + i * ld + j;
    if (j > i) *p = 0.0;
    else if (j == i) *p *= 0.5;
  }
}

// As = Abar + Abar' (n x n) from its non-zero blocks: Abar(s_a, s_b) =
// ASS(a, b), Abar(d_j, s_b) = ADS(j, b), zero elsewhere.  colidx[i] is the
// kept index of pivot i (or -1), pref[i] the kept count up to i.
__global__ void sym_scatter_kernel(const double* ASS, int64_t lss, const double* ADS,
                                   int64_t lds, const int32_t* colidx, const int32_t* pref,
                                   int64_t n, double* As, int64_t lda) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    auto abar = [&](int64_t x, int64_t y) -> double {
      const int32_t cy = colidx[y];
      if (cy < 0) return 0.0;
      const int32_t cx = colidx[x];
      if (cx >= 0) return ASS[(int64_t)cx * lss + cy];
      return ADS[(x - pref[x]) * lds + cy];
    };
    As[i * lda + j] = abar(i, j) + abar(j, i);
  }
}

}  // namespace

cudaError_t launch_pivot_lists(const uint8_t* acc, int64_t n, int32_t* pref, int32_t* sidx,
                               int32_t* didx, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  pivot_lists_kernel<<<1, 1024, 0, s>>>(acc, n, pref, sidx, didx);
  return cudaGetLastError();
}

cudaError_t launch_pattern_mask(double* Lb, int64_t ld, int64_t n, const int32_t* pref,
                                const int64_t* rdev, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  pattern_mask_kernel<<<grid_n(n * n, 256), 256, 0, s>>>(Lb, ld, n, pref, rdev);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double* src, int64_t lds, const int32_t* idx, int64_t n,
                               int count_rejected, const int64_t* rdev, double* dst, int64_t ldd,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_rows_kernel<<<grid_n(n * n, 256), 256, 0, s>>>(src, lds, idx, n, count_rejected, rdev,
                                                         dst, ldd);
  return cudaGetLastError();
}

cudaError_t launch_phi(double* P, int64_t ld, int64_t nmax, const int64_t* rdev, cudaStream_t s) {
  if (nmax <= 0) return cudaSuccess;
  phi_kernel<<<grid_n(nmax * nmax, 256), 256, 0, s>>>(P, ld, rdev);
  return cudaGetLastError();
}

cudaError_t launch_sym_scatter(const double* ASS, int64_t lss, const double* ADS, int64_t lds,
                               const int32_t* colidx, const int32_t* pref, int64_t n, double* As,
                               int64_t lda, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  sym_scatter_kernel<<<grid_n(n * n, 256), 256, 0, s>>>(ASS, lss, ADS, lds, colidx, pref, n, As,
                                                         lda);
  return cudaGetLastError();
}

}  // namespace cpinv
