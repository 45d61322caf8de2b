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

constexpr int kPanelRows = 8;
constexpr int kPanelThreads = 256;

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
// Bounded wait for *ctr >= target (one thread): false after kFlagSpinLimit
// polls (about a second), with ST_TIMEOUT recorded in *status; the caller
// goes on either way.  Later reads are ordered after the poll by a fence.
__device__ __forceinline__ bool wait_at_least(const int64_t* ctr, int64_t target, int32_t* status) {
  bool ok = false;
  for (uint32_t it = 0; it < kFlagSpinLimit; ++it) {
    if (ld_relaxed(ctr) >= target) {
      ok = true;
      break;
    }
    __nanosleep(it < 64 ? 32 : 256);
  }
  if (!ok) atomicOr(status, ST_TIMEOUT);
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return ok;
}

// The beta-bit integer that the residue planes hold for the factor entry v
// of a row with scale E, in two's complement.
__device__ __forceinline__ int64_t scaled_int(double v, int E, int beta) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int64_t m = (int64_t)crt::integerize(bits, E, beta);
  return (bits >> 63) ? -m : m;
}

// (hi:lo) += a b over 128 bits, two's complement.  |a|, |b| < 2^kMaxBeta, so
// a sum of up to kMaxLast products stays below 2^126.  The product is
// independent of the accumulator; only the carry chain is serial.
constexpr int kMaxBeta = 60;
__device__ __forceinline__ void mac128(uint64_t& lo, int64_t& hi, int64_t a, int64_t b) {
  const uint64_t plo = (uint64_t)a * (uint64_t)b;
  const int64_t phi = __mul64hi(a, b);
  asm("add.cc.u64 %0, %0, %2;\n\taddc.s64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(plo), "l"(phi));
}

// Four residues (bytes) per register.
constexpr int kRvWords = crt::kMaxMod / 4;
static_assert(crt::kMaxMod % 4 == 0, "residue packing");

// The residues of the bulk update (columns 0 .. kb) at block entry (ir, jc),
// every load in flight at once; issued before the exact sum over the last
// columns so that their latency hides behind it.
__device__ __forceinline__ void load_residues(const PanelExactParams& p, int64_t ir, int64_t jc,
                                              uint32_t (&rv)[kRvWords]) {
  const size_t plane = (size_t)p.Mpad * (size_t)p.Npad;
  const uint8_t* r = p.R + ir * p.Npad + jc;
  uint32_t b[crt::kMaxMod];
#pragma unroll
  for (int m = 0; m < crt::kMaxMod; ++m) b[m] = (p.has_bulk && m < p.n_upd) ? r[(size_t)m * plane] : 0u;
#pragma unroll
  for (int w = 0; w < kRvWords; ++w)
    rv[w] = b[4 * w] | (b[4 * w + 1] << 8) | (b[4 * w + 2] << 16) | (b[4 * w + 3] << 24);
}

// A(k0 + ir, k0 + jc) - X(ir, jc), the difference rounded once, where X is the
// exact update: the CRT value of the residues rv (columns 0 .. kb of the
// factor, when has_bulk) plus (hi:lo), the exact sum over columns kb .. k0
// formed by the caller from the factor's scaled integers.
__device__ __forceinline__ double apply_update(const PanelExactParams& p,
                                               const crt::CrtShared& sh, int shift,
                                               float inv_ptop, int64_t ir, int64_t jc,
                                               double a_old, const uint32_t (&rv)[kRvWords],
                                               uint64_t lo, int64_t hi) {
  uint32_t Y[crt::kLimbs] = {0, 0, 0, 0, 0};
  if (p.has_bulk) {
    uint64_t acc[crt::kLimbs];
#pragma unroll
    for (int l = 0; l < crt::kLimbs; ++l) acc[l] = 0;
#pragma unroll
    for (int m = 0; m < crt::kMaxMod; ++m) {
      if (m >= p.n_upd) break;
      const uint32_t t = sh.tab[m][(rv[m >> 2] >> (8 * (m & 3))) & 0xFFu];
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

__global__ void __launch_bounds__(kPanelThreads, 4) chol_panel_exact_kernel(PanelExactParams p) {
  const int64_t n = eval_dim(p.nd, p.rdev);
  const int64_t k0 = p.k0;
  if (k0 >= n) return;
  const int bw = (int)((n - k0) < p.b ? (n - k0) : p.b);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = k0 + bw + (int64_t)(blockIdx.x - 1) * kPanelRows;
  const bool helper = p.has_update && blockIdx.x >= 1 && (int)blockIdx.x <= p.helpers;
  if (blockIdx.x > 0 && row0 >= n && !helper) return;  // nothing for this CTA
  __shared__ crt::CrtShared sh;
  // CTA 0 factors the diagonal block; the other CTAs solve their rows
  // against it: the two phases' shared memory is one
  __shared__ union {
    chol::DiagScratch diag;
    struct {
      double Ts[32][33];
      double dv[32];
    } rows;
  } u;
  double(&Ts)[32][33] = u.rows.Ts;
  double* dv = u.rows.dv;
  __shared__ int64_t Lt[kMaxLast][32];  // Lt[k][j]: scaled integer of L(k0 + j, kb + k)
  __shared__ int go;
  double* A = p.A;
  const int64_t lda = p.lda;
  int shift = 0;
  float inv_ptop = 0.f;
  if (p.has_update) {
    // the block's rows over the last columns kb .. k0 as scaled integers
    // (Lt[k][j] for L(k0 + j, kb + k)) and the CRT tables; every global load
    // is issued before the first is used
    constexpr int kLtPer = kMaxLast * 32 / kPanelThreads;
    double lv[kLtPer];
    int le[kLtPer];
#pragma unroll
    for (int q = 0; q < kLtPer; ++q) {
      const int e = threadIdx.x + kPanelThreads * q, k = e >> 5, j = e & 31;
      const bool in = k < p.k_last && j < bw;
      lv[q] = in ? A[(k0 + j) * lda + p.kb + k] : 0.0;
      le[q] = in ? p.E[k0 + j] : 0;
    }
    if (p.has_bulk) {
      const crt::Consts& c = p.consts[p.n_upd];
      constexpr int kTabPer = (crt::kMaxMod * 32 + kPanelThreads - 1) / kPanelThreads;
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&c.tab[0][0]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sh.tab[0][0]);
      uint32_t tv[kTabPer];
#pragma unroll
      for (int q = 0; q < kTabPer; ++q) {
        const int e = threadIdx.x + kPanelThreads * q;
        tv[q] = e < p.n_upd * 32 ? src[e] : 0u;
      }
      const int em = threadIdx.x;
      const uint32_t mv = em < p.n_upd * crt::kLimbs ? c.Mj[em / crt::kLimbs][em % crt::kLimbs] : 0u;
      uint32_t pv = 0, hv = 0;
      if (threadIdx.x < crt::kLimbs) {
        pv = c.P[threadIdx.x];
        hv = c.halfP[threadIdx.x];
      }
      shift = c.shift;
      inv_ptop = c.inv_ptop;
#pragma unroll
      for (int q = 0; q < kTabPer; ++q) {
        const int e = threadIdx.x + kPanelThreads * q;
        if (e < p.n_upd * 32) dst[e] = tv[q];
      }
      if (em < p.n_upd * crt::kLimbs) sh.Mj[em / crt::kLimbs][em % crt::kLimbs] = mv;
      if (threadIdx.x < crt::kLimbs) {
        sh.P[threadIdx.x] = pv;
        sh.halfP[threadIdx.x] = hv;
      }
    }
#pragma unroll
    for (int q = 0; q < kLtPer; ++q) {
      const int e = threadIdx.x + kPanelThreads * q, k = e >> 5, j = e & 31;
      if (k < kMaxLast) Lt[k][j] = scaled_int(lv[q], le[q], p.beta);
    }
    __syncthreads();
  }
  // The exact update of the block's entries [beg, end) of its lower
  // triangle, four lanes per entry: lane g of a quad loads the residues of
  // the moduli g, g + 4, ..., sums the columns kb + g, kb + g + 4, ... and the
  // CRT terms of its moduli; the partial sums meet by shuffles and lane 0
  // centres, rounds and stores.  The loop is warp-uniform (idle quads work on
  // a repeated entry and store nothing) so the shuffles see the whole warp.
  auto block_update_quads = [&](int beg, int end) {
    const int g = threadIdx.x & 3;
    constexpr int kQuads = kPanelThreads / 4;
    constexpr int kModPerLane = crt::kMaxMod / 4;
    for (int base = beg; base < end; base += kQuads) {
      const int o0 = base + (int)(threadIdx.x >> 2);
      const bool valid = o0 < end;
      int i, j;
      tri_index(valid ? o0 : beg, i, j);
      double* a = A + (k0 + i) * lda + (k0 + j);
      const double a_old = g == 0 ? *a : 0.0;
      uint32_t rv[kModPerLane];
      const size_t plane = (size_t)p.Mpad * (size_t)p.Npad;
      const uint8_t* rp = p.R + (int64_t)i * p.Npad + j;
#pragma unroll
      for (int t = 0; t < kModPerLane; ++t) {
        const int m = g + 4 * t;
        rv[t] = (p.has_bulk && m < p.n_upd) ? rp[(size_t)m * plane] : 0u;
      }
      uint64_t lo = 0;
      int64_t hi = 0;
#pragma unroll 4
      for (int k = g; k < p.k_last; k += 4) mac128(lo, hi, Lt[k][i], Lt[k][j]);
      uint64_t acc[crt::kLimbs] = {0, 0, 0, 0, 0};
      if (p.has_bulk) {
#pragma unroll
        for (int t = 0; t < kModPerLane; ++t) {
          const int m = g + 4 * t;
          if (m < p.n_upd) {
            const uint32_t tv = sh.tab[m][rv[t]];
#pragma unroll
            for (int l = 0; l < crt::kLimbs; ++l) acc[l] += (uint64_t)tv * sh.Mj[m][l];
          }
        }
      }
#pragma unroll
      for (int off = 1; off < 4; off <<= 1) {
        const uint64_t plo = __shfl_xor_sync(0xffffffffu, lo, off);
        const int64_t phi = __shfl_xor_sync(0xffffffffu, hi, off);
        lo += plo;
        hi += phi + (lo < plo ? 1 : 0);
#pragma unroll
        for (int l = 0; l < crt::kLimbs; ++l) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], off);
      }
      if (g == 0 && valid) {
        uint32_t Y[crt::kLimbs] = {0, 0, 0, 0, 0};
        if (p.has_bulk) {
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
        const int scale = p.E[k0 + i] - 1022 - p.beta + p.E[k0 + j] - 1022 - p.beta;
        *a = fma(1.0, a_old, -crt::limbs_to_double(Y, scale));
      }
    }
  };
  const int tri = bw * (bw + 1) / 2;
  if (helper) {
    // this CTA's share of the diagonal block's update, then count it
    const int chunk = (tri + p.helpers - 1) / p.helpers;
    const int beg = ((int)blockIdx.x - 1) * chunk;
    const int end = beg + chunk < tri ? beg + chunk : tri;
    block_update_quads(beg, end);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((unsigned long long*)&p.st->diag_count, 1ull);
    if (row0 >= n) return;
  }
  if (blockIdx.x == 0) {
    // the diagonal block: update (lower part), factor, publish, residues
    if (p.has_update && p.helpers == 0) {
      block_update_quads(0, tri);
      __syncthreads();
    } else if (p.has_update) {
      // wait for the helpers' shares (bounded; ST_TIMEOUT on expiry)
      if (threadIdx.x == 0) wait_at_least(&p.st->diag_count, p.diag_target, &p.st->status);
      __syncthreads();
    }
    if (warp < chol::kDiagWarps)
      chol::diag_chol_block(A, lda, p.nd, k0, p.b, p.st, p.rdev, p.accepted, p.dinv, p.spd,
                            u.diag);
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
    // this row's scaled integers over the last columns, lane k holding k and
    // k + 32; lane c sums against column c of the block
    const double a_old = lane < bw ? A[i * lda + k0 + lane] : 0.0;
    uint32_t rv[kRvWords];
    load_residues(p, i - k0, lane < bw ? lane : 0, rv);
    int64_t ai[kMaxLast / 32];
#pragma unroll
    for (int q = 0; q < kMaxLast / 32; ++q) {
      const int k = lane + 32 * q;
      ai[q] = k < p.k_last ? scaled_int(A[i * lda + p.kb + k], p.E[i], p.beta) : 0;
    }
    uint64_t lo = 0;
    int64_t hi = 0;
#pragma unroll
    for (int q = 0; q < kMaxLast / 32; ++q) {
      const int kend = p.k_last - 32 * q < 32 ? p.k_last - 32 * q : 32;
#pragma unroll 4
      for (int kk = 0; kk < kend; ++kk) {
        const int64_t a = __shfl_sync(0xffffffffu, ai[q], kk);
        mac128(lo, hi, a, Lt[32 * q + kk][lane]);
      }
    }
    if (lane < bw) acc = apply_update(p, sh, shift, inv_ptop, i - k0, lane, a_old, rv, lo, hi);
  } else if (row_ok && lane < bw) {
    acc = A[i * lda + k0 + lane];
  }
  if (threadIdx.x == 0) go = wait_at_least(&p.st->panel_flag, p.epoch, &p.st->status);
  __syncthreads();
  if (!go) return;
  // Ts[r][c] = T(r, c) / T(c, c) below the diagonal (see panel_solve_rows);
  // L2 loads (the block was written by another CTA in this launch), all in
  // one round trip, scaled in shared memory afterwards
  if (threadIdx.x < 32) dv[threadIdx.x] = threadIdx.x < bw ? __ldcg(p.dinv + threadIdx.x) : 0.0;
  for (int e = threadIdx.x; e < 32 * 32; e += kPanelThreads) {
    const int r = e >> 5, c = e & 31;
    Ts[r][c] = (r < bw && c < r) ? __ldcg(A + (k0 + r) * lda + (k0 + c)) : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += kPanelThreads) Ts[e >> 5][e & 31] *= dv[e & 31];
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

// The panel kernel's bounded wait on a counter that nothing advances: it
// must give up, record ST_TIMEOUT and return (the failure path of every
// flag wait, exercised without a fault).
__global__ void wait_selftest_kernel(DevState* st) {
  if (threadIdx.x == 0) wait_at_least(&st->spare[0], 1, &st->status);
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
  if (p.k_last < 0 || p.k_last > kMaxLast || (p.has_update && p.kb + p.k_last != p.k0) ||
      p.beta < 1 || p.beta > kMaxBeta)
    return cudaErrorInvalidValue;
  const int64_t ctas = chol_panel_exact_ctas(p.nd.max, p.k0, p.b);
  if (p.helpers < 0 || p.helpers >= ctas) return cudaErrorInvalidValue;
  // The panel kernel shares its SMs with the look-ahead residue product on
  // another stream; with the largest shared-memory carveout an SM running
  // panel CTAs still takes a product CTA (the carveout of a busy SM cannot
  // change, so a small one would keep the product off those SMs).
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(chol_panel_exact_kernel,
                                         cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  chol_panel_exact_kernel<<<(unsigned)ctas, kPanelThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(DevState* st, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_rowscale(const double* A, int64_t lda, Dim nd, const int64_t* rdev,
                            int64_t rows_max, int32_t* E, cudaStream_t s) {
  rowscale_kernel<<<grid1d(rows_max, 256), 256, 0, s>>>(A, lda, nd, rdev, rows_max, E);
  return cudaGetLastError();
}


}  // namespace cpinv
