// FP64 matrix product on the CUDA cores (DFMA), the "plain FP64" arithmetic.
//
// C = alpha * op(A) op(B) + beta * C, row-major operands, optional lower-only
// output (for the symmetric products G'G, L'L, A - L L').  On GB300 the FP64
// pipe issues about two DFMA per clock per SM (1.2 TFLOP/s over 152 SMs), so
// this kernel is bound by that pipe at any reasonable tile shape: a 64 x 64
// tile per 256-thread CTA with 4 x 4 outputs per thread keeps the shared-memory
// and DRAM traffic far below what the DFMA rate can consume.
#include "common.cuh"
#include "kernels.h"

namespace cpinv {

namespace {

constexpr int TK = 16;

// T x T output tile per 256-thread CTA, (T/16) x (T/16) outputs per thread.
// T = 64 for large outputs; 32 and 16 spread small products over more SMs
// (each SM's FP64 pipe is narrow, so a product must occupy many SMs).
template <bool TA, bool TB, int T>
__global__ void __launch_bounds__(256) dgemm_kernel(GemmParams p) {
  constexpr int U = T / 16;
  if (blockIdx.z) {
    int64_t z = blockIdx.z, zo = 0;
    if (p.nzi > 1) {
      zo = z / p.nzi;
      z -= zo * p.nzi;
    }
    p.A += z * p.zA + zo * p.oA;
    p.B += z * p.zB + zo * p.oB;
    p.C += z * p.zC + zo * p.oC;
    p.M.off += z * p.zM;
    p.N.off += z * p.zN;
    p.K.off += z * p.zK;
    p.rdev += z * p.zR + zo * p.oR;
  }
  const int64_t M = eval_dim(p.M, p.rdev);
  const int64_t N = eval_dim(p.N, p.rdev);
  const int64_t K = eval_dim(p.K, p.rdev);
  const int64_t i0 = (int64_t)blockIdx.y * T;
  const int64_t j0 = (int64_t)blockIdx.x * T;
  if (i0 >= M || j0 >= N) return;
  if (p.lower && j0 > i0 + T - 1) return;  // tile strictly above the diagonal

  __shared__ double As[TK][T + 1];
  __shared__ double Bs[TK][T + 1];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[U][U];
#pragma unroll
  for (int a = 0; a < U; ++a)
#pragma unroll
    for (int b = 0; b < U; ++b) acc[a][b] = 0.0;

  for (int64_t k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
    for (int q = 0; q < (T * TK) / 256; ++q) {
      const int e = tid + 256 * q;
      int i, k;
      if (TA) { k = e / T; i = e % T; } else { i = e / TK; k = e % TK; }
      const int64_t gi = i0 + i, gk = k0 + k;
      double v = 0.0;
      if (gi < M && gk < K) v = TA ? p.A[gk * p.lda + gi] : p.A[gi * p.lda + gk];
      As[k][i] = v;
    }
#pragma unroll
    for (int q = 0; q < (T * TK) / 256; ++q) {
      const int e = tid + 256 * q;
      int j, k;
      if (TB) { j = e / TK; k = e % TK; } else { k = e / T; j = e % T; }
      const int64_t gj = j0 + j, gk = k0 + k;
      double v = 0.0;
      if (gj < N && gk < K) v = TB ? p.B[gj * p.ldb + gk] : p.B[gk * p.ldb + gj];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      double a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = As[k][ty + 16 * u];
#pragma unroll
      for (int u = 0; u < U; ++u) b[u] = Bs[k][tx + 16 * u];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t gi = i0 + ty + 16 * u;
    if (gi >= M) continue;
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int64_t gj = j0 + tx + 16 * v;
      if (gj >= N) continue;
      if (p.lower && gj > gi) continue;
      double* c = p.C + gi * p.ldc + gj;
      double out = p.alpha * acc[u][v];
      if (p.beta != 0.0) out = fma(p.beta, *c, out);
      *c = out;
    }
  }
}

// Narrow outputs (N <= NC <= 16, no aliasing, whole matrix): a CTA owns 64
// rows and every column of C, four threads per row each summing a quarter of
// the K range for all NC columns (partial sums met by shuffles), so that no
// FP64 instruction computes a padding column -- with the 64 x 64 tiles a
// product of 4 columns would spend 15 of every 16 FMAs on padding.
constexpr int kSkRows = 64, kSkK = 32;
template <bool TA, bool TB, int NC>
__global__ void __launch_bounds__(256) dgemm_skinny_kernel(GemmParams p) {
  if (blockIdx.z) {
    int64_t z = blockIdx.z, zo = 0;
    if (p.nzi > 1) {
      zo = z / p.nzi;
      z -= zo * p.nzi;
    }
    p.A += z * p.zA + zo * p.oA;
    p.B += z * p.zB + zo * p.oB;
    p.C += z * p.zC + zo * p.oC;
    p.M.off += z * p.zM;
    p.N.off += z * p.zN;
    p.K.off += z * p.zK;
    p.rdev += z * p.zR + zo * p.oR;
  }
  const int64_t M = eval_dim(p.M, p.rdev);
  const int64_t N = eval_dim(p.N, p.rdev);
  const int64_t K = eval_dim(p.K, p.rdev);
  const int64_t i0 = (int64_t)blockIdx.y * kSkRows;
  if (i0 >= M || N <= 0) return;
  __shared__ double As[kSkK][kSkRows + 1];
  __shared__ double Bs[kSkK][NC];
  const int tid = threadIdx.x;
  const int r = tid >> 2, sub = tid & 3;
  double acc[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += kSkK) {
#pragma unroll
    for (int q = 0; q < (kSkRows * kSkK) / 256; ++q) {
      const int e = tid + 256 * q;
      int i, k;
      if (TA) { k = e / kSkRows; i = e % kSkRows; } else { i = e / kSkK; k = e % kSkK; }
      const int64_t gi = i0 + i, gk = k0 + k;
      double v = 0.0;
      if (gi < M && gk < K) v = TA ? p.A[gk * p.lda + gi] : p.A[gi * p.lda + gk];
      As[k][i] = v;
    }
    for (int e = tid; e < kSkK * NC; e += 256) {
      int j, k;
      if (TB) { j = e / kSkK; k = e % kSkK; } else { k = e / NC; j = e % NC; }
      const int64_t gk = k0 + k;
      double v = 0.0;
      if (j < N && gk < K) v = TB ? p.B[j * p.ldb + gk] : p.B[gk * p.ldb + j];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = sub; kk < kSkK; kk += 4) {
      const double a = As[kk][r];
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] = fma(a, Bs[kk][j], acc[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 1);
    acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 2);
  }
  const int64_t gi = i0 + r;
  if (sub != 0 || gi >= M) return;
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    if (j >= N) break;
    double* c = p.C + gi * p.ldc + j;
    double out = p.alpha * acc[j];
    if (p.beta != 0.0) out = fma(p.beta, *c, out);
    *c = out;
  }
}

template <int NC>
cudaError_t launch_skinny(const GemmParams& p, bool transA, bool transB, cudaStream_t s) {
  dim3 grid(1u, (unsigned)((p.M.max + kSkRows - 1) / kSkRows), (unsigned)(p.nz > 1 ? p.nz : 1));
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  if (!transA && !transB) dgemm_skinny_kernel<false, false, NC><<<grid, 256, 0, s>>>(p);
  else if (!transA && transB) dgemm_skinny_kernel<false, true, NC><<<grid, 256, 0, s>>>(p);
  else if (transA && !transB) dgemm_skinny_kernel<true, false, NC><<<grid, 256, 0, s>>>(p);
  else dgemm_skinny_kernel<true, true, NC><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

template <int T>
cudaError_t launch_tile(const GemmParams& p, bool transA, bool transB, cudaStream_t s) {
  dim3 grid((unsigned)((p.N.max + T - 1) / T), (unsigned)((p.M.max + T - 1) / T),
            (unsigned)(p.nz > 1 ? p.nz : 1));
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  if (!transA && !transB) dgemm_kernel<false, false, T><<<grid, 256, 0, s>>>(p);
  else if (!transA && transB) dgemm_kernel<false, true, T><<<grid, 256, 0, s>>>(p);
  else if (transA && !transB) dgemm_kernel<true, false, T><<<grid, 256, 0, s>>>(p);
  else dgemm_kernel<true, true, T><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dgemm(const GemmParams& p, bool transA, bool transB, cudaStream_t s) {
  const int64_t Mmax = p.M.max, Nmax = p.N.max;
  if (Mmax <= 0 || Nmax <= 0) return cudaSuccess;
  if (p.pad) {
    // C aliases an operand: every CTA must own whole rows of C (all N columns),
    // so that it reads them completely before it overwrites them.
    if (Nmax <= 16) return launch_tile<16>(p, transA, transB, s);
    if (Nmax <= 32) return launch_tile<32>(p, transA, transB, s);
    if (Nmax <= 64) return launch_tile<64>(p, transA, transB, s);
    return cudaErrorInvalidValue;
  }
  const int64_t nz = p.nz > 1 ? p.nz : 1;
  // narrow outputs over enough rows to fill the GPU (with few rows and a
  // long K the tiled kernel's more, smaller CTAs spread the FP64 work wider)
  if (Nmax <= 16 && !p.lower && nz * ((Mmax + kSkRows - 1) / kSkRows) >= 152) {
    if (Nmax <= 4) return launch_skinny<4>(p, transA, transB, s);
    if (Nmax <= 8) return launch_skinny<8>(p, transA, transB, s);
    return launch_skinny<16>(p, transA, transB, s);
  }
  auto tiles = [&](int64_t t) { return nz * ((Mmax + t - 1) / t) * ((Nmax + t - 1) / t); };
  if (tiles(64) >= 152 || (Mmax >= 64 && Nmax >= 64 && tiles(32) > 4 * 152))
    return launch_tile<64>(p, transA, transB, s);
  if (tiles(32) >= 152) return launch_tile<32>(p, transA, transB, s);
  return launch_tile<16>(p, transA, transB, s);
}

}  // namespace cpinv
