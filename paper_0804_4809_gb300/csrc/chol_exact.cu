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

#include "chol_device.cuh"
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

// One launch per panel of the exact-slice factorisation: the panel's update
// (the CRT reconstruction of the exact residue product of the factor's
// earlier columns), the factorisation of the diagonal block, the solve of
// the rows below it and their residue split, fused.
//  * CTAs 1..helpers first apply the update to a share of the diagonal
//    block's lower triangle each and count their share done (atomic add to
//    the call's state).
//  * CTA 0 waits for that count (or applies the update itself when there
//    are no helpers), factors the block on four warps, publishes it (release
//    store of the panel's number into the call's state), then writes the
//    block's residues.
//  * Every CTA but 0 applies the update to its eight rows (one warp per row,
//    lane c = column c), waits for the publication, and solves its rows by
//    forward substitution against the published block.
// Every wait is bounded: on expiry the CTA records ST_TIMEOUT and goes on.
// The grid is small (at most 1 + n/8 CTAs of 256 threads, four resident per
// SM), so every CTA is resident at once; no CTA waits on one that waits.
constexpr uint32_t kFlagSpinLimit = 1u << 22;
constexpr int kMaxLast = 64;  // columns of the update summed in the panel kernel itself

// The waiters poll with relaxed loads (an acquire load per poll would
// invalidate the SM's L1 each time, slowing every CTA on that SM, the
// publishing one included) and order their later reads with one fence.
__device__ __forceinline__ int64_t ld_relaxed(const int64_t* p) {
  int64_t v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int64_t* p, int64_t v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Signed magnitude of the beta-bit integer that the residue planes hold for
// the factor entry v of a row with scale E (sign in bit 63).
__device__ __forceinline__ uint64_t scaled_int(double v, int E, int beta) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  return crt::integerize(bits, E, beta) | (bits & 0x8000000000000000ull);
}

// acc += a b for signed-magnitude integers below 2^62 (acc two's complement
// over 128 bits: sums of up to 64 such products fit).
__device__ __forceinline__ void mac128(uint64_t& lo, int64_t& hi, uint64_t a, uint64_t b) {
  const uint64_t ma = a & 0x7FFFFFFFFFFFFFFFull, mb = b & 0x7FFFFFFFFFFFFFFFull;
  const uint64_t plo = ma * mb, phi = __umul64hi(ma, mb);
  if ((a ^ b) >> 63) {
    const uint64_t r = lo - plo;
    hi -= (int64_t)(phi + (r > lo ? 1u : 0u));
    lo = r;
  } else {
    const uint64_t r = lo + plo;
    hi += (int64_t)(phi + (r < plo ? 1u : 0u));
    lo = r;
  }
}

// A(k0 + ir, k0 + jc) - X(ir, jc), the difference rounded once, where X is the
// exact update: the CRT value of the residues in R (columns 0 .. kb of the
// factor, when has_bulk) plus (hi:lo), the exact sum over columns kb .. k0
// formed by the caller from the factor's scaled integers.
__device__ __forceinline__ double apply_update(const PanelExactParams& p,
                                               const crt::CrtShared& sh, int shift,
                                               float inv_ptop, int64_t ir, int64_t jc,
                                               double a_old, uint64_t lo, int64_t hi) {
  uint32_t Y[crt::kLimbs] = {0, 0, 0, 0, 0};
  if (p.has_bulk) {
    const size_t plane = (size_t)p.Mpad * (size_t)p.Npad;
    const uint8_t* r = p.R + ir * p.Npad + jc;
    // every residue load in flight at once: one memory latency per output
    uint32_t rv[crt::kMaxMod];
#pragma unroll
    for (int m = 0; m < crt::kMaxMod; ++m) rv[m] = m < p.n_upd ? r[(size_t)m * plane] : 0u;
    uint64_t acc[crt::kLimbs];
#pragma unroll
    for (int l = 0; l < crt::kLimbs; ++l) acc[l] = 0;
#pragma unroll
    for (int m = 0; m < crt::kMaxMod; ++m) {
      if (m >= p.n_upd) break;
      const uint32_t t = sh.tab[m][rv[m]];
#pragma unroll
      for (int l = 0; l < crt::kLimbs; ++l) acc[l] += (uint64_t)t * sh.Mj[m][l];
    }
    uint32_t S[crt::kLimbs];
    uint64_t carry = 0;
#pragma unroll
    for (int l = 0; l < crt::kLimbs; ++l) {
      const uint64_t v = acc[l] + carry;
      S[l] = (uint32_t)v;
      carry = v >> 32;
    }
    crt::crt_centre(S, sh.P, sh.halfP, shift, inv_ptop, Y);
  }
  crt::limbs_add128(Y, lo, hi);
  const int scale = p.E[p.k0 + ir] - 1022 - p.beta + p.E[p.k0 + jc] - 1022 - p.beta;
  const double x = crt::limbs_to_double(Y, scale);
  return fma(1.0, a_old, -x);
}

__device__ __forceinline__ void split_store(const PanelExactParams& p, int64_t row, int64_t col,
                                            double l) {
  const uint64_t bits = (uint64_t)__double_as_longlong(l);
  const uint64_t a = crt::integerize(bits, p.E[row], p.beta);
  crt::store_residues(a, (bits >> 63) != 0, p.n_mod, p.RL + (size_t)row * p.rl_kpad + col,
                      (size_t)p.rl_rows * (size_t)p.rl_kpad);
}

// Entry o of the lower triangle of the block, o = i (i + 1) / 2 + j.
__device__ __forceinline__ void tri_index(int o, int& i, int& j) {
  i = (int)((sqrtf(8.0f * (float)o + 1.0f) - 1.0f) * 0.5f);
  if ((i + 1) * (i + 2) / 2 <= o) ++i;
  if (i * (i + 1) / 2 > o) --i;
  j = o - i * (i + 1) / 2;
}

__global__ void __launch_bounds__(256, 4) chol_panel_exact_kernel(PanelExactParams p) {
  const int64_t n = eval_dim(p.nd, p.rdev);
  const int64_t k0 = p.k0;
  if (k0 >= n) return;
  const int bw = (int)((n - k0) < p.b ? (n - k0) : p.b);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = k0 + bw + (int64_t)(blockIdx.x - 1) * kPanelRows;
  const bool helper = p.has_update && blockIdx.x >= 1 && (int)blockIdx.x <= p.helpers;
  if (blockIdx.x > 0 && row0 >= n && !helper) return;  // nothing for this CTA
  __shared__ crt::CrtShared sh;
  __shared__ double Ts[32][33];
  __shared__ double dv[32];
  __shared__ uint64_t Lt[kMaxLast][32];  // Lt[k][j]: scaled integer of L(k0 + j, kb + k)
  __shared__ int go;
  double* A = p.A;
  const int64_t lda = p.lda;
  int shift = 0;
  float inv_ptop = 0.f;
  if (p.has_update) {
    if (p.has_bulk) {
      const crt::Consts& c = p.consts[p.n_upd];
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&c.tab[0][0]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sh.tab[0][0]);
      for (int e = threadIdx.x; e < p.n_upd * 32; e += blockDim.x) dst[e] = src[e];
      for (int e = threadIdx.x; e < p.n_upd * crt::kLimbs; e += blockDim.x)
        sh.Mj[e / crt::kLimbs][e % crt::kLimbs] = c.Mj[e / crt::kLimbs][e % crt::kLimbs];
      if (threadIdx.x < crt::kLimbs) {
        sh.P[threadIdx.x] = c.P[threadIdx.x];
        sh.halfP[threadIdx.x] = c.halfP[threadIdx.x];
      }
      shift = c.shift;
      inv_ptop = c.inv_ptop;
    }
    // the block's rows over the last columns kb .. k0, as scaled integers
    for (int e = threadIdx.x; e < p.k_last * 32; e += blockDim.x) {
      const int k = e >> 5, j = e & 31;
      Lt[k][j] = j < bw ? scaled_int(A[(k0 + j) * lda + p.kb + k], p.E[k0 + j], p.beta) : 0ull;
    }
    __syncthreads();
  }
  // the exact update of block entry (i, j): CRT part + sum over the last columns
  auto block_update = [&](int i, int j) {
    uint64_t lo = 0;
    int64_t hi = 0;
    for (int k = 0; k < p.k_last; ++k) mac128(lo, hi, Lt[k][i], Lt[k][j]);
    double* a = A + (k0 + i) * lda + (k0 + j);
    *a = apply_update(p, sh, shift, inv_ptop, i, j, *a, lo, hi);
  };
  const int tri = bw * (bw + 1) / 2;
  if (helper) {
    // this CTA's share of the diagonal block's update, then count it
    const int chunk = (tri + p.helpers - 1) / p.helpers;
    const int beg = ((int)blockIdx.x - 1) * chunk;
    const int end = beg + chunk < tri ? beg + chunk : tri;
    for (int o = beg + threadIdx.x; o < end; o += blockDim.x) {
      int i, j;
      tri_index(o, i, j);
      block_update(i, j);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((unsigned long long*)&p.st->diag_count, 1ull);
    if (row0 >= n) return;
  }
  if (blockIdx.x == 0) {
    // the diagonal block: update (lower part), factor, publish, residues
    if (p.has_update && p.helpers == 0) {
      for (int o = threadIdx.x; o < tri; o += blockDim.x) {
        int i, j;
        tri_index(o, i, j);
        block_update(i, j);
      }
      __syncthreads();
    } else if (p.has_update) {
      // wait for the helpers' shares (bounded; ST_TIMEOUT on expiry)
      if (threadIdx.x == 0) {
        int ok = 0;
        for (uint32_t it = 0; it < kFlagSpinLimit; ++it) {
          if (ld_relaxed(&p.st->diag_count) >= p.diag_target) {
            ok = 1;
            break;
          }
          __nanosleep(it < 64 ? 32 : 256);
        }
        if (!ok) atomicOr(&p.st->status, ST_TIMEOUT);
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
      }
      __syncthreads();
    }
    if (warp < chol::kDiagWarps)
      chol::diag_chol_block(A, lda, p.nd, k0, p.b, p.st, p.rdev, p.accepted, p.dinv, p.spd);
    // publish the block (factor and 1/T_cc written by warps 0-3) ...
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release(&p.st->panel_flag, p.epoch);
    // ... then its residues, while the other CTAs solve their rows
    for (int o = threadIdx.x; o < tri; o += blockDim.x) {
      int i, j;
      tri_index(o, i, j);
      split_store(p, k0 + i, k0 + j, A[(k0 + i) * lda + (k0 + j)]);
    }
    return;
  }
  // rows below the block: the update first, then wait for the block
  const int64_t i = row0 + warp;
  const bool row_ok = i < n;
  double acc = 0.0;
  if (row_ok && p.has_update) {
    // this row's scaled integers over the last columns, lane k holding k,
    // k + 32, k + 64; lane c sums against column c of the block
    uint64_t ai[kMaxLast / 32];
#pragma unroll
    for (int q = 0; q < kMaxLast / 32; ++q) {
      const int k = lane + 32 * q;
      ai[q] = k < p.k_last ? scaled_int(A[i * lda + p.kb + k], p.E[i], p.beta) : 0ull;
    }
    uint64_t lo = 0;
    int64_t hi = 0;
#pragma unroll
    for (int q = 0; q < kMaxLast / 32; ++q) {
      const int kend = p.k_last - 32 * q < 32 ? p.k_last - 32 * q : 32;
      for (int kk = 0; kk < kend; ++kk) {
        const uint64_t a = __shfl_sync(0xffffffffu, ai[q], kk);
        mac128(lo, hi, a, Lt[32 * q + kk][lane]);
      }
    }
    if (lane < bw) acc = apply_update(p, sh, shift, inv_ptop, i - k0, lane, A[i * lda + k0 + lane], lo, hi);
  } else if (row_ok && lane < bw) {
    acc = A[i * lda + k0 + lane];
  }
  if (threadIdx.x == 0) {
    int ok = 0;
    for (uint32_t it = 0; it < kFlagSpinLimit; ++it) {
      if (ld_relaxed(&p.st->panel_flag) >= p.epoch) {
        ok = 1;
        break;
      }
      __nanosleep(it < 64 ? 32 : 256);
    }
    if (!ok) atomicOr(&p.st->status, ST_TIMEOUT);
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    go = ok;
  }
  __syncthreads();
  if (!go) return;
  // Ts[r][c] = T(r, c) / T(c, c) below the diagonal (see panel_solve_rows);
  // L2 loads (the block was written by another CTA in this launch), all in
  // one round trip, scaled in shared memory afterwards
  if (threadIdx.x < 32) dv[threadIdx.x] = threadIdx.x < bw ? __ldcg(p.dinv + threadIdx.x) : 0.0;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    Ts[r][c] = (r < bw && c < r) ? __ldcg(A + (k0 + r) * lda + (k0 + c)) : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) Ts[e >> 5][e & 31] *= dv[e & 31];
  __syncthreads();
  if (!row_ok) return;
  for (int c = 0; c < bw; ++c) {
    const double ac = __shfl_sync(0xffffffffu, acc, c);
    if (lane > c) acc = fma(-ac, Ts[lane][c], acc);
  }
  if (lane < bw) {
    const double l = acc * dv[lane];
    A[i * lda + k0 + lane] = l;
    split_store(p, i, k0 + lane, l);
  }
}

inline unsigned grid1d(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 8) g = 152 * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

int64_t chol_panel_exact_ctas(int64_t nmax, int64_t k0, int b) {
  const int64_t below = nmax - k0 - b;
  return 1 + (below > 0 ? (below + kPanelRows - 1) / kPanelRows : 0);
}

cudaError_t launch_chol_panel_exact(const PanelExactParams& p, cudaStream_t s) {
  if (p.b > 32 || p.b < 1 || (p.has_bulk && (!p.consts || !p.R))) return cudaErrorInvalidValue;
  if (p.k_last < 0 || p.k_last > kMaxLast || (p.has_update && p.kb + p.k_last != p.k0))
    return cudaErrorInvalidValue;
  const int64_t ctas = chol_panel_exact_ctas(p.nd.max, p.k0, p.b);
  if (p.helpers < 0 || p.helpers >= ctas) return cudaErrorInvalidValue;
  chol_panel_exact_kernel<<<(unsigned)ctas, 256, 0, s>>>(p);
  return cudaGetLastError();
}

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
