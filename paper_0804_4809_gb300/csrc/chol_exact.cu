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

constexpr int kPanelRows = 8;       // rows per CTA below block kn
constexpr int kBlockRows = 4;       // rows per CTA of block kn
constexpr int kPanelThreads = 256;

// One launch per panel of the exact-slice factorisation, pipelined by one
// block: launch p solves the rows below the diagonal block of panel p
// (factored by the previous launch) and factors the diagonal block of panel
// p + 1, so that the rows' work runs beside the next block's pivots instead
// of after them.  With ks = k0 of panel p and kn = ks + b:
//  * CTAs 1..nbr solve the rows of block kn against block ks (four rows
//    each, one warp per row), count themselves done (st->panel_flag), then
//    write those rows' residues.
//  * CTAs nbr+1..nbr+helpers update block kn's lower triangle, one entry per
//    quad: the CRT value of the bulk residues (columns 0 .. kb, the
//    look-ahead product) and the exact sum over the columns kb .. ks first,
//    then, once the block rows are solved, the exact sum over panel p's
//    columns, all added and the difference rounded once; they count
//    themselves done (st->diag_count) and then write the residues of block
//    ks's entries.
//  * CTA 0 waits for that count and factors block kn on four warps.
//  * The other CTAs take the rows below block kn: solve against block ks,
//    residues, then the same once-rounded update of their entries in panel
//    p + 1's columns.
// The first launch of a factorisation (one CTA) factors block 0 only.
// Every wait is bounded: on expiry the CTA records ST_TIMEOUT and goes on.
// CTA 0 waits on the helpers and the rest on CTAs 1..nbr only, all of them
// low-numbered CTAs of a grid of at most 1 + 8 + 9 + n/8 CTAs of 256
// threads; no waited-on CTA waits on a higher-numbered one.
constexpr uint32_t kFlagSpinLimit = 1u << 22;
constexpr int kMaxLast = 96;  // columns of an update summed in the panel kernel itself

// The waiters poll with relaxed loads (an acquire load per poll would
// invalidate the SM's L1 each time, slowing every CTA on that SM) and order
// their later reads with one fence.
__device__ __forceinline__ int64_t ld_relaxed(const int64_t* p) {
  int64_t v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
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

// Counts this CTA done on *ctr once all its threads' global writes are
// visible device-wide.
__device__ __forceinline__ void count_done(int64_t* ctr) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd((unsigned long long*)ctr, 1ull);
}

// The beta-bit integer that the residue planes hold for the factor entry v
// of a row with scale E, in two's complement.
__device__ __forceinline__ int64_t scaled_int(double v, int E, int beta) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int64_t m = (int64_t)crt::integerize(bits, E, beta);
  return (bits >> 63) ? -m : m;
}

// (hi:lo) += a b over 128 bits, two's complement.  |a|, |b| < 2^kMaxBeta, so
// a sum of up to kMaxLast products stays below 2^(2 kMaxBeta + 6.6) < 2^127.
// The product is independent of the accumulator; only the carry chain is
// serial.
constexpr int kMaxBeta = 60;
static_assert(2 * kMaxBeta + 7 <= 127, "exact sums over kMaxLast columns fit in 128 bits");
__device__ __forceinline__ void mac128(uint64_t& lo, int64_t& hi, int64_t a, int64_t b) {
  const uint64_t plo = (uint64_t)a * (uint64_t)b;
  const int64_t phi = __mul64hi(a, b);
  asm("add.cc.u64 %0, %0, %2;\n\taddc.s64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(plo), "l"(phi));
}

// Four residues (bytes) per register.
constexpr int kRvWords = crt::kMaxMod / 4;
static_assert(crt::kMaxMod % 4 == 0, "residue packing");

// The residues of the bulk update (columns 0 .. kb) at entry (ir, jc) of the
// update's output (rows from kn), every load in flight at once.
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

// 2^-scale of the exact update of entry (row, col): both rows' factor
// entries are beta-bit integers at their rows' scales.
__device__ __forceinline__ int update_scale(const PanelExactParams& p, int64_t row, int64_t col) {
  return p.E[row] - 1022 - p.beta + p.E[col] - 1022 - p.beta;
}

// a_old - X rounded once, where X is the exact update of entry (row, col):
// the CRT value of the residues rv (columns 0 .. kb, when has_bulk) plus
// (hi:lo), the exact sum over the columns kb .. kn.
__device__ __forceinline__ double apply_update(const PanelExactParams& p,
                                               const crt::CrtShared& sh, int shift,
                                               float inv_ptop, int64_t row, int64_t col,
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
  return fma(1.0, a_old, -crt::limbs_to_double(Y, update_scale(p, row, col)));
}

__device__ __forceinline__ void split_store(const PanelExactParams& p, int64_t row, int64_t col,
                                            double l) {
  const uint64_t bits = (uint64_t)__double_as_longlong(l);
  const uint64_t a = crt::integerize(bits, p.E[row], p.beta);
  crt::store_residues(a, (bits >> 63) != 0, p.n_mod, p.RL + (size_t)row * p.rl_kpad + col,
                      (size_t)p.rl_rows * (size_t)p.rl_kpad);
}

// Entry o of the lower triangle of a block, o = i (i + 1) / 2 + j.
__device__ __forceinline__ void tri_index(int o, int& i, int& j) {
  i = (int)((sqrtf(8.0f * (float)o + 1.0f) - 1.0f) * 0.5f);
  if ((i + 1) * (i + 2) / 2 <= o) ++i;
  if (i * (i + 1) / 2 > o) --i;
  j = o - i * (i + 1) / 2;
}

// The CRT constants of the update's moduli into shared memory (every thread
// of the CTA; the caller synchronises).
__device__ __forceinline__ void load_tables(const PanelExactParams& p, crt::CrtShared& sh,
                                            int& shift, float& inv_ptop) {
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

// Lt[k][j] for k0 <= k < k1: the scaled integer of L(kn + j, kb + k), the
// rows of block kn over the columns kb .. kn (L2 loads: panel p's part is
// written by other CTAs of this launch).  Consecutive threads read
// consecutive columns of a row; the row stride of Lt is odd in 8-byte words,
// so those stores spread over the banks.  The caller synchronises.
constexpr int kLtStride = 33;
__device__ __forceinline__ void load_lt(const PanelExactParams& p,
                                        int64_t (&Lt)[kMaxLast][kLtStride], int bwn, int k0,
                                        int k1) {
  const int w = k1 - k0;
  if (w <= 0) return;
  const int total = w * 32;
  // four loads per thread in flight at a time
  constexpr int kPer = 4;
  for (int base = 0; base < total; base += kPer * kPanelThreads) {
    double v[kPer];
    int ev[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = base + (int)threadIdx.x + kPanelThreads * q;
      const int j = e / w, k = k0 + (e - j * w);
      const bool in = e < total && j < bwn;
      v[q] = in ? __ldcg(p.A + (p.kn + j) * p.lda + p.kb + k) : 0.0;
      ev[q] = in ? p.E[p.kn + j] : 0;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = base + (int)threadIdx.x + kPanelThreads * q;
      if (e < total) {
        const int j = e / w, k = k0 + (e - j * w);
        Lt[k][j] = scaled_int(v[q], ev[q], p.beta);
      }
    }
  }
}

// Block ks (factored by the previous launch) for the forward substitution:
// dv = 1/T(c, c), Ts[r][c] = T(r, c) / T(c, c) below the diagonal.  The
// caller synchronises before and after the scaling step below.
__device__ __forceinline__ void load_block(const PanelExactParams& p, double (&Ts)[32][33],
                                           double* dv) {
  const int b = p.b;
  const double d = threadIdx.x < b ? __ldcg(p.dinv_prev + threadIdx.x) : 0.0;
  constexpr int kPer = 32 * 32 / kPanelThreads;
  double t[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = (int)threadIdx.x + kPanelThreads * q, r = e >> 5, c = e & 31;
    t[q] = (r < b && c < r) ? __ldcg(p.A + (p.ks + r) * p.lda + (p.ks + c)) : 0.0;
  }
  if (threadIdx.x < 32) dv[threadIdx.x] = d;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = (int)threadIdx.x + kPanelThreads * q;
    Ts[e >> 5][e & 31] = t[q];
  }
}
__device__ __forceinline__ void scale_block(double (&Ts)[32][33], const double* dv) {
  for (int e = threadIdx.x; e < 32 * 32; e += kPanelThreads) Ts[e >> 5][e & 31] *= dv[e & 31];
}
// Forward substitution of one row (lane c holds column c) against block ks;
// returns L(i, ks + lane).
__device__ __forceinline__ double solve_row(double acc, const double (&Ts)[32][33],
                                            const double* dv, int b) {
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < b; ++c) {
    const double ac = __shfl_sync(0xffffffffu, acc, c);
    if (lane > c) acc = fma(-ac, Ts[lane][c], acc);
  }
  return acc * dv[lane];
}

__global__ void __launch_bounds__(kPanelThreads, 3) chol_panel_exact_kernel(PanelExactParams p) {
  const int64_t n = eval_dim(p.nd, p.rdev);
  const int64_t ks = p.ks, kn = p.kn;
  const int b = p.b;
  // order of block kn (0: past the end)
  const int bwn = kn < n ? (int)((n - kn) < b ? (n - kn) : b) : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x = (int)blockIdx.x;
  const int first_helper = 1 + p.nbr, first_row = 1 + p.nbr + p.helpers;
  __shared__ crt::CrtShared sh;
  // CTA 0 factors block kn, the row CTAs solve against block ks: the two
  // phases' shared memory is one
  __shared__ union {
    chol::DiagScratch diag;
    struct {
      double Ts[32][33];
      double dv[32];
    } rows;
  } u;
  __shared__ int64_t Lt[kMaxLast][kLtStride];
  double* A = p.A;
  const int64_t lda = p.lda;

  if (x == 0) {
    // block kn: wait for its update, then factor
    if (bwn == 0) return;
    if (p.has_update) {
      if (threadIdx.x == 0) wait_at_least(&p.st->diag_count, p.diag_target, &p.st->status);
      __syncthreads();
    }
    if (warp < chol::kDiagWarps)
      chol::diag_chol_block(A, lda, p.nd, kn, b, p.st, p.rdev, p.accepted, p.dinv_next, p.spd,
                            u.diag);
    return;
  }

  if (x < first_helper) {
    // the rows of block kn against block ks, then count
    const int64_t i = kn + (int64_t)(x - 1) * kBlockRows + warp;
    const bool row_ok = warp < kBlockRows && i < kn + bwn;
    const double acc = (row_ok && lane < b) ? A[i * lda + ks + lane] : 0.0;
    load_block(p, u.rows.Ts, u.rows.dv);
    __syncthreads();
    scale_block(u.rows.Ts, u.rows.dv);
    __syncthreads();
    double l = 0.0;
    if (row_ok) {
      l = solve_row(acc, u.rows.Ts, u.rows.dv, b);
      if (lane < b) A[i * lda + ks + lane] = l;
    }
    count_done(&p.st->panel_flag);
    // their residues, off the path that others wait on
    if (row_ok && lane < b) split_store(p, i, ks + lane, l);
    return;
  }

  int shift = 0;
  float inv_ptop = 0.f;
  if (x < first_row) {
    // block kn's update: entry o = h * 64 + quad of its lower triangle
    const int h = x - first_helper;
    const int tri = bwn * (bwn + 1) / 2;
    const int g = threadIdx.x & 3;
    const int o = h * (kPanelThreads / 4) + (int)(threadIdx.x >> 2);
    const bool valid = o < tri;
    int bi = 0, bj = 0;
    if (valid) tri_index(o, bi, bj);
    const double a_old = (valid && g == 0) ? A[(kn + bi) * lda + (kn + bj)] : 0.0;
    constexpr int kModPerLane = crt::kMaxMod / 4;
    uint32_t rv[kModPerLane];
    {
      const size_t plane = (size_t)p.Mpad * (size_t)p.Npad;
      const uint8_t* rp = p.R + (int64_t)bi * p.Npad + bj;
#pragma unroll
      for (int t = 0; t < kModPerLane; ++t) {
        const int m = g + 4 * t;
        rv[t] = (p.has_bulk && m < p.n_upd && tri > 0) ? rp[(size_t)m * plane] : 0u;
      }
    }
    // the columns kb .. ks (final before this launch) of the block rows
    const int ko = (int)(ks - p.kb);
    if (p.has_bulk && tri > 0) load_tables(p, sh, shift, inv_ptop);
    load_lt(p, Lt, bwn, 0, ko);
    __syncthreads();
    // the bulk part: lane g sums the CRT terms of the moduli g, g + 4, ...;
    // the quad's partial sums meet by shuffles and lane 0 centres them
    uint32_t Y[crt::kLimbs] = {0, 0, 0, 0, 0};
    if (p.has_bulk) {
      uint64_t acc[crt::kLimbs] = {0, 0, 0, 0, 0};
#pragma unroll
      for (int t = 0; t < kModPerLane; ++t) {
        const int m = g + 4 * t;
        if (m < p.n_upd) {
          const uint32_t tv = sh.tab[m][rv[t]];
#pragma unroll
          for (int l = 0; l < crt::kLimbs; ++l) acc[l] += (uint64_t)tv * sh.Mj[m][l];
        }
      }
#pragma unroll
      for (int off = 1; off < 4; off <<= 1)
#pragma unroll
        for (int l = 0; l < crt::kLimbs; ++l) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], off);
      if (g == 0 && valid) {
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
    }
    // plus the exact sum over the columns kb .. ks now, and over panel p's
    // columns once the block rows are solved
    uint64_t lo = 0;
    int64_t hi = 0;
#pragma unroll 4
    for (int k = g; k < ko; k += 4) mac128(lo, hi, Lt[k][bi], Lt[k][bj]);
    if (threadIdx.x == 0) wait_at_least(&p.st->panel_flag, p.rows_target, &p.st->status);
    __syncthreads();
    load_lt(p, Lt, bwn, ko, p.k_last);
    __syncthreads();
#pragma unroll 4
    for (int k = ko + g; k < p.k_last; k += 4) mac128(lo, hi, Lt[k][bi], Lt[k][bj]);
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      const uint64_t plo = __shfl_xor_sync(0xffffffffu, lo, off);
      const int64_t phi = __shfl_xor_sync(0xffffffffu, hi, off);
      lo += plo;
      hi += phi + (lo < plo ? 1 : 0);
    }
    if (g == 0 && valid) {
      crt::limbs_add128(Y, lo, hi);
      A[(kn + bi) * lda + (kn + bj)] =
          fma(1.0, a_old, -crt::limbs_to_double(Y, update_scale(p, kn + bi, kn + bj)));
    }
    count_done(&p.st->diag_count);
    // then the residues of block ks's own entries (factored by the previous
    // launch), a share per helper
    if (ks >= 0 && ks < n) {
      const int bws = (int)((n - ks) < b ? (n - ks) : b);
      const int tri_s = bws * (bws + 1) / 2;
      const int chunk = (tri_s + p.helpers - 1) / p.helpers;
      const int end = (h + 1) * chunk < tri_s ? (h + 1) * chunk : tri_s;
      for (int e = h * chunk + (int)threadIdx.x; e < end; e += kPanelThreads) {
        int i, j;
        tri_index(e, i, j);
        split_store(p, ks + i, ks + j, A[(ks + i) * lda + (ks + j)]);
      }
    }
    return;
  }

  // rows below block kn: solve against block ks, then their update in panel
  // p + 1's columns
  const int64_t row0 = kn + b + (int64_t)(x - first_row) * kPanelRows;
  if (row0 >= n) return;  // nothing for this CTA (uniform)
  const int64_t i = row0 + warp;
  const bool row_ok = i < n;
  // every global load of the row issued first
  const double acc0 = (row_ok && lane < b) ? A[i * lda + ks + lane] : 0.0;
  const double a_old = (row_ok && lane < bwn) ? A[i * lda + kn + lane] : 0.0;
  uint32_t rv[kRvWords];
  load_residues(p, row_ok ? i - kn : 0, lane < bwn ? lane : 0, rv);
  constexpr int kQ = kMaxLast / 32;
  double vold[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int64_t col = p.kb + lane + 32 * q;
    vold[q] = (row_ok && col < ks && col - p.kb < p.k_last) ? A[i * lda + col] : 0.0;
  }
  const int ko = (int)(ks - p.kb);  // columns kb .. ks: final before this launch
  if (p.has_bulk) load_tables(p, sh, shift, inv_ptop);
  load_block(p, u.rows.Ts, u.rows.dv);
  load_lt(p, Lt, bwn, 0, ko);
  __syncthreads();
  scale_block(u.rows.Ts, u.rows.dv);
  __syncthreads();
  double l = 0.0;
  if (row_ok) {
    l = solve_row(acc0, u.rows.Ts, u.rows.dv, b);
    if (lane < b) {
      A[i * lda + ks + lane] = l;
      split_store(p, i, ks + lane, l);
    }
  }
  // this row's scaled integers over the columns kb .. kn, lane k holding
  // k, k + 32, k + 64; panel p's entries come from the solve just done
  int64_t ai[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int64_t col = p.kb + lane + 32 * q;
    const double vn = __shfl_sync(0xffffffffu, l, (int)((col - ks) & 31));
    const double v = col >= ks ? vn : vold[q];
    ai[q] = (row_ok && col - p.kb < p.k_last) ? scaled_int(v, p.E[i], p.beta) : 0;
  }
  // the exact sum: lane c against column c of the block, over the columns
  // [k0, k1) of kb .. kn (warp-uniform loops), in two independent chains
  uint64_t lo = 0, lo2 = 0;
  int64_t hi = 0, hi2 = 0;
  auto mac_range = [&](int k0, int k1) {
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int kbeg = k0 > 32 * q ? k0 : 32 * q;
      const int kend = k1 < 32 * q + 32 ? k1 : 32 * q + 32;
      int k = kbeg;
      for (; k + 1 < kend; k += 2) {
        const int64_t a0 = __shfl_sync(0xffffffffu, ai[q], k - 32 * q);
        const int64_t a1 = __shfl_sync(0xffffffffu, ai[q], k + 1 - 32 * q);
        mac128(lo, hi, a0, Lt[k][lane]);
        mac128(lo2, hi2, a1, Lt[k + 1][lane]);
      }
      if (k < kend) {
        const int64_t a0 = __shfl_sync(0xffffffffu, ai[q], k - 32 * q);
        mac128(lo, hi, a0, Lt[k][lane]);
      }
    }
  };
  mac_range(0, ko);
  // panel p's columns of the block rows, once they are solved
  if (threadIdx.x == 0) wait_at_least(&p.st->panel_flag, p.rows_target, &p.st->status);
  __syncthreads();
  load_lt(p, Lt, bwn, ko, p.k_last);
  __syncthreads();
  mac_range(ko, p.k_last);
  lo += lo2;
  hi += hi2 + (lo < lo2 ? 1 : 0);
  if (row_ok && lane < bwn)
    A[i * lda + kn + lane] = apply_update(p, sh, shift, inv_ptop, i, kn + lane, a_old, rv, lo, hi);
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

int chol_panel_exact_nbr(int b) { return (b + kBlockRows - 1) / kBlockRows; }
int chol_panel_exact_helpers(int b) { return (b * (b + 1) / 2 + kPanelThreads / 4 - 1) / (kPanelThreads / 4); }

int64_t chol_panel_exact_ctas(int64_t nmax, int64_t kn, int b) {
  const int64_t below = nmax - kn - b;
  return 1 + chol_panel_exact_nbr(b) + chol_panel_exact_helpers(b) +
         (below > 0 ? (below + kPanelRows - 1) / kPanelRows : 0);
}

cudaError_t launch_chol_panel_exact(const PanelExactParams& p, cudaStream_t s) {
  if (p.b > 32 || p.b < 1 || !p.dinv_next)
    return cudaErrorInvalidValue;
  int64_t ctas = 1;  // the first launch: CTA 0 factors block 0
  if (p.has_update) {
    if ((p.has_bulk && (!p.consts || !p.R)) || !p.dinv_prev || p.ks < 0 || p.kn != p.ks + p.b ||
        p.k_last < 0 || p.k_last > kMaxLast || p.kb + p.k_last != p.kn || p.beta < 1 ||
        p.beta > kMaxBeta || p.nbr != chol_panel_exact_nbr(p.b) ||
        p.helpers != chol_panel_exact_helpers(p.b))
      return cudaErrorInvalidValue;
    ctas = chol_panel_exact_ctas(p.nd.max, p.kn, p.b);
  } else if (p.kn != 0) {
    return cudaErrorInvalidValue;
  }
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
