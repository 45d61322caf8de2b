// Gaussian radial-basis design matrices on the GPU (Sec. 1 and Sec. 4 of the
// paper: W = G+ F trains the output weights of an RBF network), and the
// normal equations A = G'G, B = G'F formed from the inputs X, the centres C
// and the width w without G ever being stored:
//
//   G_ij = exp(-|x_i - c_j|^2 / (2 w^2)),  |x_i - c_j|^2 summed over the d
//   coordinates in order, (x - c)^2 accumulated by FMAs, in FP64.
//
// cpinv_rbf_design writes G (m x n, FP64) to HBM.
// cpinv_rbf_normal_equations: A and B in the exact-slice arithmetic of the
// library, with the residue split of op(A) = G' fused into the generation:
//   1. rbf_bound_kernel: per centre j, a lower bound of min_i |x_i - c_j|^2
//      in FP32, hence an upper bound of the biased exponent of max_i G_ij (at
//      most one above it), the row scale of G' in the residue planes;
//   2. rbf_split_kernel: per K chunk (rows of X), G' generated tile by tile
//      in FP64 and cut straight into its residue planes (no FP64 G in HBM);
//   3. the tensor-core residue products G'G (lower) and G'F, and the CRT
//      reconstruction, as for any exact product (gemm_crt.cu).
// One chunk of at most 4096 rows of X is exact and rounded once; chunks are
// added in FP64, as the exact product of the library does for long K.
#include <cmath>
#include <cstring>
#include <utility>

#include "../../include/cpinv.h"
#include "common.cuh"
#include "crt.h"
#include "crt_device.cuh"
#include "kernels.h"

namespace cpinv {
namespace {

constexpr int kMaxD = CPINV_RBF_MAX_D;
constexpr int kRbfBeta = 62;      // integer bits of G' in its residue planes (as the Gram's)
constexpr int kRbfBetaF = 53;     // integer bits of F
constexpr int64_t kChunk = 4096;  // exactness bound of one residue product (K)

__device__ __forceinline__ bool finite_bits(uint64_t b) { return ((b >> 52) & 0x7FF) != 0x7FF; }

// G_ij from coordinates in shared memory (xs: this data row, cs: this
// centre, both contiguous over the d coordinates).
__device__ __forceinline__ double rbf_value(const double* xs, const double* cs, int d,
                                            double inv2w2) {
  double d2 = 0.0;
  for (int k = 0; k < d; ++k) {
    const double t = xs[k] - cs[k];
    d2 = fma(t, t, d2);
  }
  return exp(-(d2 * inv2w2));
}

// G (m x n, row-major, ld ldg): tiles of 64 data rows x 32 centres, thread
// (tx, ty) computes column j0 + tx for rows i0 + ty + 8q (coalesced stores).
__global__ void __launch_bounds__(256) rbf_design_kernel(const double* X, int64_t m, int d,
                                                         int64_t ldx, const double* C, int64_t n,
                                                         int64_t ldc, double inv2w2, double* G,
                                                         int64_t ldg) {
  __shared__ double xs[64][kMaxD + 1];
  __shared__ double cs[32][kMaxD + 1];
  const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 32;
  for (int e = threadIdx.x; e < 64 * d; e += 256) {
    const int r = e / d, k = e - r * d;
    xs[r][k] = i0 + r < m ? X[(i0 + r) * ldx + k] : 0.0;
  }
  for (int e = threadIdx.x; e < 32 * d; e += 256) {
    const int r = e / d, k = e - r * d;
    cs[r][k] = j0 + r < n ? C[(j0 + r) * ldc + k] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t j = j0 + tx;
  if (j >= n) return;
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    const int r = ty + 8 * q;
    if (i0 + r >= m) break;
    G[(i0 + r) * ldg + j] = rbf_value(xs[r], cs[tx], d, inv2w2);
  }
}

// Per centre j: dmin[j] = bits of a lower bound of min_i |x_i - c_j|^2 (FP32,
// non-negative, so the bit patterns order like the values; atomicMin into an
// array preset to a huge value), and the non-finite flag of X and C.  The
// FP32 sum is lowered by 2^-20 (d2 + sum (|x| + |c|)^2), four times its
// rounding error bound (2^-22 of that: the conversions of x and c, the
// difference, the squares and the sum), so it bounds the FP64 value.
// Grid: x over centres (32 per block, one per lane), y over chunks of rows.
__global__ void __launch_bounds__(256) rbf_bound_kernel(const double* X, int64_t m, int d,
                                                        int64_t ldx, const double* C, int64_t n,
                                                        int64_t ldc, uint32_t* dmin,
                                                        int32_t* status) {
  __shared__ float xs[64][kMaxD + 1];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  float c[kMaxD];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kMaxD; ++k) {
    double v = (j < n && k < d) ? C[j * ldc + k] : 0.0;
    if (!isfinite(v)) {
      bad = true;
      v = 0.0;
    }
    c[k] = (float)v;
  }
  float best = INFINITY;
  const int64_t rows_per = (m + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = r0 + rows_per < m ? r0 + rows_per : m;
  for (int64_t b = r0; b < r1; b += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * d; e += 256) {
      const int r = e / d, k = e - r * d;
      double v = b + r < r1 ? X[(b + r) * ldx + k] : 0.0;
      if (!isfinite(v)) {
        bad = true;
        v = 0.0;
      }
      xs[r][k] = (float)v;
    }
    __syncthreads();
    const int rows = (int)(r1 - b < 64 ? r1 - b : 64);
    for (int r = wy; r < rows; r += 8) {
      float d2 = 0.f, s = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxD; ++k) {
        if (k >= d) break;
        const float t = xs[r][k] - c[k];
        const float a = fabsf(xs[r][k]) + fabsf(c[k]);
        d2 = fmaf(t, t, d2);
        s = fmaf(a, a, s);
      }
      const float lb = fmaxf(0.f, d2 - 9.5367431640625e-07f * (d2 + s));  // 2^-20
      best = fminf(best, lb);
    }
  }
  if (j < n && best < INFINITY) atomicMin(&dmin[j], __float_as_uint(best));
  if (bad) atomicOr(status, ST_NONFINITE);
}

// E[j] >= the biased exponent of max_i G_ij (by at most one): with y =
// exp(-dmin / (2 w^2)), floor(log2 y) = floor(-dmin log2(e) / (2 w^2)), taken
// in FP32 with a 2^-8 margin (above the rounding of the product and of the
// FP64 exponential near a power of two); 0 when every G_ij underflows.
__global__ void rbf_expo_kernel(const uint32_t* dmin, int64_t n, float inv2w2_log2e,
                                int64_t rows_max, int32_t* E) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= rows_max) return;
  int e = 0;
  if (j < n) {
    const float dm = __uint_as_float(dmin[j]);
    if (dm == 0.f) {
      e = 1023;  // a centre on a data point: max G = 1
    } else {
      const float t = -dm * inv2w2_log2e;  // log2 of the largest G_ij
      const float f = floorf(t + 0.00390625f);
      e = (f >= -1100.f) ? 1023 + (int)fminf(f, 0.f) : 0;  // NaN and underflow: 0
      if (e < 0) e = 0;
    }
  }
  E[j] = e;
}

// Residues of eight adjacent columns of one row as one 16-byte store per
// modulus (eight BF16).
template <int J>
__device__ __forceinline__ void store8(const uint32_t (&c)[8][3], int n_mod, uint4* dst,
                                       size_t plane_vec) {
  if (J >= n_mod) return;
  uint32_t w[4];
#pragma unroll
  for (int h = 0; h < 4; ++h)
    w[h] = crt::residue_pair_bf16<J>(c[2 * h][0], c[2 * h][1], c[2 * h][2], c[2 * h + 1][0],
                                     c[2 * h + 1][1], c[2 * h + 1][2], 0u);
  dst[J * plane_vec] = make_uint4(w[0], w[1], w[2], w[3]);
}
template <int... Js>
__device__ __forceinline__ void store8_all(std::integer_sequence<int, Js...>,
                                           const uint32_t (&c)[8][3], int n_mod, uint4* dst,
                                           size_t plane_vec) {
  (store8<Js>(c, n_mod, dst, plane_vec), ...);
}

// Residue planes S[j][row][k] of op(A) = G' over the data rows i0 .. i0 +
// kuse (k = i - i0): row = centre j, scale E[j], beta bits; every G_ij is
// positive, so the integers are non-negative.  Tiles of 32 centres x 64 data
// rows; thread (q, g): centre q, data rows 8g .. 8g + 7.
__global__ void __launch_bounds__(256) rbf_split_kernel(const double* X, int64_t i0, int64_t kuse,
                                                        int d, int64_t ldx, const double* C,
                                                        int64_t n, int64_t ldc, double inv2w2,
                                                        const int32_t* E, int64_t rows_max,
                                                        int64_t kpad, int n_mod, int beta,
                                                        __nv_bfloat16* out, int32_t* status) {
  __shared__ double xs[64][kMaxD + 1];
  __shared__ double cs[32][kMaxD + 1];
  const int64_t c0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * d; e += 256) {
    const int r = e / d, k = e - r * d;
    xs[r][k] = k0 + r < kuse ? X[(i0 + k0 + r) * ldx + k] : 0.0;
  }
  for (int e = threadIdx.x; e < 32 * d; e += 256) {
    const int r = e / d, k = e - r * d;
    cs[r][k] = c0 + r < n ? C[(c0 + r) * ldc + k] : 0.0;
  }
  __syncthreads();
  const int q = threadIdx.x >> 3, g = threadIdx.x & 7;
  const int64_t row = c0 + q;
  if (row >= rows_max) return;
  const int Er = row < n ? E[row] : 0;
  uint32_t c[8][3];
  bool over = false;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int r = 8 * g + u;
    uint64_t a = 0;
    if (row < n && k0 + r < kuse) {
      const uint64_t b = (uint64_t)__double_as_longlong(rbf_value(xs[r], cs[q], d, inv2w2));
      // the bound must cover every entry (else the integer would not fit
      // in beta bits): checked, and reported as a numerical failure
      if ((int)((b >> 52) & 0x7FF) > Er) over = true;
      else if (finite_bits(b)) a = crt::integerize(b, Er, beta);
    }
    c[u][0] = (uint32_t)(a & 0x1FFFFF);
    c[u][1] = (uint32_t)((a >> 21) & 0x1FFFFF);
    c[u][2] = (uint32_t)(a >> 42);
  }
  if (over) atomicOr(status, ST_NUMERICAL);
  uint4* dst = reinterpret_cast<uint4*>(out + (size_t)row * kpad + k0 + 8 * g);
  store8_all(std::make_integer_sequence<int, crt::kMaxMod>{}, c, n_mod, dst,
             (size_t)rows_max * (size_t)kpad / 8);
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Workspace layout of cpinv_rbf_normal_equations.
struct RbfLayout {
  int n_mod, n_modf;
  int64_t kc, kpad, mpad, npad, fpad;
  size_t off_state, off_dmin, off_EA, off_EB, off_SA, off_SB, off_R, total;
};

RbfLayout rbf_layout(int64_t m, int64_t n, int64_t k) {
  RbfLayout L{};
  L.kc = m < kChunk ? (m > 0 ? m : 1) : kChunk;
  L.n_mod = crt_moduli_for(L.kc, kRbfBeta, kRbfBeta);
  L.n_modf = crt_moduli_for(L.kc, kRbfBeta, kRbfBetaF);
  const int64_t bk = crt_block_k(), bm = crt_block_m();
  L.kpad = round_up(L.kc, bk);
  L.mpad = round_up(n > 0 ? n : 1, bm);    // centres: rows of G'
  L.npad = round_up(n > 0 ? n : 1, 256);   // columns of the Gram's residues
  L.fpad = round_up(k > 0 ? k : 1, 256);   // columns of F (rows of its N x K view)
  size_t b = 0;
  auto take = [&](size_t x) {
    b = (b + 1023) / 1024 * 1024;
    const size_t at = b;
    b += x;
    return at;
  };
  L.off_state = take(sizeof(DevState));
  L.off_dmin = take(sizeof(uint32_t) * (size_t)L.mpad);
  L.off_EA = take(sizeof(int32_t) * (size_t)L.mpad);
  L.off_EB = take(sizeof(int32_t) * (size_t)L.fpad);
  L.off_SA = take(2 * (size_t)L.n_mod * (size_t)L.mpad * (size_t)L.kpad);
  L.off_SB = take(2 * (size_t)L.n_modf * (size_t)L.fpad * (size_t)L.kpad);
  const size_t r_gram = (size_t)L.n_mod * (size_t)L.mpad * (size_t)L.npad;
  const size_t r_f = (size_t)L.n_modf * (size_t)L.mpad * (size_t)L.fpad;
  L.off_R = take(r_gram > r_f ? r_gram : r_f);
  L.total = b + 256;
  return L;
}

#define RBF_CK(x)                                   \
  do {                                              \
    cudaError_t _e = (x);                           \
    if (_e != cudaSuccess) return CPINV_ERR_CUDA;   \
  } while (0)

int check_rbf_args(const double* X, int64_t m, int64_t d, int64_t ldx, const double* C, int64_t n,
                   int64_t ldc, double width) {
  if (m < 0 || n < 0 || d < 0 || ldx < d || ldc < d) return CPINV_ERR_INVALID_ARG;
  if (d > kMaxD) return CPINV_ERR_UNSUPPORTED;
  if (!(width > 0.0) || !std::isfinite(width)) return CPINV_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && ((d > 0 && (!X || !C)))) return CPINV_ERR_INVALID_ARG;
  return CPINV_OK;
}

}  // namespace
}  // namespace cpinv

using namespace cpinv;

extern "C" {

int cpinv_rbf_design(const double* X, int64_t m, int64_t d, int64_t ldx, const double* C,
                     int64_t n, int64_t ldc, double width, double* G, int64_t ldg, void* stream) {
  if (int rc = check_rbf_args(X, m, d, ldx, C, n, ldc, width)) return rc;
  if (ldg < n) return CPINV_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return CPINV_OK;
  if (!G) return CPINV_ERR_INVALID_ARG;
  if ((m + 63) / 64 > 65535) return CPINV_ERR_UNSUPPORTED;
  const double inv2w2 = 1.0 / (2.0 * width * width);
  cudaStream_t s = (cudaStream_t)stream;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 63) / 64));
  KernelTimer t;
  RBF_CK(t.run(KT_AUX, s, [&] {
    rbf_design_kernel<<<grid, 256, 0, s>>>(X, m, (int)d, ldx, C, n, ldc, inv2w2, G, ldg);
    return cudaGetLastError();
  }));
  return CPINV_OK;
}

size_t cpinv_rbf_normal_equations_workspace_size(int64_t m, int64_t n, int64_t d, int64_t k) {
  if (m < 0 || n < 0 || d < 0 || k < 0 || d > kMaxD) return 0;
  return rbf_layout(m, n, k).total;
}

int cpinv_rbf_normal_equations(const double* X, int64_t m, int64_t d, int64_t ldx, const double* C,
                               int64_t n, int64_t ldc, double width, const double* F, int64_t k,
                               int64_t ldf, double* A, int64_t lda, double* B, int64_t ldb,
                               void* workspace, size_t workspace_bytes, int32_t check,
                               void* stream) {
  if (int rc = check_rbf_args(X, m, d, ldx, C, n, ldc, width)) return rc;
  if (k < 0 || lda < n || (F && (ldf < k || !B || ldb < k))) return CPINV_ERR_INVALID_ARG;
  if (n == 0) return CPINV_OK;
  if (!A) return CPINV_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const bool with_f = F && k > 0;
  if (m == 0) {
    // no data: A = 0, B = 0
    RBF_CK(cudaMemset2DAsync(A, (size_t)lda * sizeof(double), 0, (size_t)n * sizeof(double),
                             (size_t)n, s));
    if (with_f)
      RBF_CK(cudaMemset2DAsync(B, (size_t)ldb * sizeof(double), 0, (size_t)k * sizeof(double),
                               (size_t)n, s));
    return CPINV_OK;
  }
  const RbfLayout L = rbf_layout(m, n, with_f ? k : 0);
  if (L.n_mod < 0 || L.n_modf < 0) return CPINV_ERR_UNSUPPORTED;
  if (!workspace || ((uintptr_t)workspace & 255u) || workspace_bytes < L.total)
    return CPINV_ERR_WORKSPACE;
  if (L.kpad / 64 > 65535 || L.mpad / 32 > 65535) return CPINV_ERR_UNSUPPORTED;
  char* w = (char*)workspace;
  DevState* st = (DevState*)(w + L.off_state);
  uint32_t* dmin = (uint32_t*)(w + L.off_dmin);
  int32_t* EA = (int32_t*)(w + L.off_EA);
  int32_t* EB = (int32_t*)(w + L.off_EB);
  __nv_bfloat16* SA = (__nv_bfloat16*)(w + L.off_SA);
  __nv_bfloat16* SB = (__nv_bfloat16*)(w + L.off_SB);
  uint8_t* R = (uint8_t*)(w + L.off_R);
  const double inv2w2 = 1.0 / (2.0 * width * width);
  const float inv2w2_log2e = (float)(inv2w2 * 1.4426950408889634);
  if (!crt_consts_device()) return CPINV_ERR_CUDA;
  RBF_CK(cudaMemsetAsync(st, 0, sizeof(DevState), s));
  RBF_CK(cudaMemsetAsync(dmin, 0x7F, sizeof(uint32_t) * (size_t)L.mpad, s));  // > +inf bits: unset
  KernelTimer t;
  // 1. row scales of G' (per centre)
  RBF_CK(t.run(KT_SPLIT, s, [&] {
    const unsigned gy = (unsigned)((m + 1023) / 1024 < 64 ? (m + 1023) / 1024 : 64);
    rbf_bound_kernel<<<dim3((unsigned)((n + 31) / 32), gy), 256, 0, s>>>(X, m, (int)d, ldx, C, n,
                                                                         ldc, dmin, &st->status);
    if (cudaGetLastError() != cudaSuccess) return cudaGetLastError();
    rbf_expo_kernel<<<(unsigned)((L.mpad + 255) / 256), 256, 0, s>>>(dmin, n, inv2w2_log2e,
                                                                     L.mpad, EA);
    return cudaGetLastError();
  }));
  const Dim Nd = hdim(n), Kd = hdim(k);
  for (int64_t i0 = 0; i0 < m; i0 += kChunk) {
    const int64_t kuse = m - i0 < kChunk ? m - i0 : kChunk;
    const double acc = i0 == 0 ? 0.0 : 1.0;  // chunks after the first add to A and B
    // 2. G' of this chunk straight into its residue planes
    RBF_CK(t.run(KT_SPLIT, s, [&] {
      dim3 grid((unsigned)(L.kpad / 64), (unsigned)(L.mpad / 32));
      rbf_split_kernel<<<grid, 256, 0, s>>>(X, i0, kuse, (int)d, ldx, C, n, ldc, inv2w2, EA,
                                            L.mpad, L.kpad, L.n_mod, kRbfBeta, SA, &st->status);
      return cudaGetLastError();
    }));
    // 3. A (+)= G'G, lower triangle
    GemmParams fl;
    std::memset(&fl, 0, sizeof(fl));
    fl.M = Nd;
    fl.N = Nd;
    fl.K = hdim(kuse);
    fl.lower = 1;
    fl.rdev = &st->rank;
    RBF_CK(crt_mma(SA, L.mpad, 0, SA, L.mpad, 0, L.kpad, kuse, L.n_mod, Nd, Nd, &st->rank, 1, R,
                   L.mpad, L.npad, &st->status, s, &t, &fl));
    RBF_CK(crt_reconstruct(R, L.mpad, L.npad, Nd, Nd, &st->rank, EA, EA, kRbfBeta, kRbfBeta, 1.0,
                           acc, A, lda, 1, L.n_mod, s, &t));
    if (!with_f) continue;
    // B (+)= G'F: F's rows of this chunk split as usual (its N x K view)
    RBF_CK(cudaMemsetAsync(EB, 0, sizeof(int32_t) * (size_t)L.fpad, s));
    const double* Fc = F + i0 * ldf;
    RBF_CK(crt_row_exponents(Fc, ldf, 1, Kd, hdim(kuse), &st->rank, L.fpad, EB, st, s, &t));
    RBF_CK(crt_split(Fc, ldf, 1, Kd, hdim(kuse), &st->rank, L.fpad, L.kpad, EB, L.n_modf,
                     kRbfBetaF, SB, s, &t));
    GemmParams fb = fl;
    fb.N = Kd;
    fb.lower = 0;
    RBF_CK(crt_mma(SA, L.mpad, 0, SB, L.fpad, 0, L.kpad, kuse, L.n_modf, Nd, Kd, &st->rank, 0, R,
                   L.mpad, L.fpad, &st->status, s, &t, &fb));
    RBF_CK(crt_reconstruct(R, L.mpad, L.fpad, Nd, Kd, &st->rank, EA, EB, kRbfBeta, kRbfBetaF, 1.0,
                           acc, B, ldb, 0, L.n_modf, s, &t));
  }
  RBF_CK(trace_finish(s, &st->rank));
  if (!check) return CPINV_OK;
  DevState h;
  RBF_CK(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
  RBF_CK(cudaStreamSynchronize(s));
  if (h.status & ST_NONFINITE) return CPINV_ERR_NONFINITE_INPUT;
  if (h.status & ST_NUMERICAL) return CPINV_ERR_NUMERICAL;
  if (h.status & ST_TIMEOUT) return CPINV_ERR_TIMEOUT;
  return CPINV_OK;
}

}  // extern "C"
