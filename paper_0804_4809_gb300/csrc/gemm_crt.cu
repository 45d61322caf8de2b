// FP64-accurate matrix products on the BF16 tensor cores (tcgen05) by residue
// arithmetic -- the "exact-slice" arithmetic of the library (see crt.h).
//
//   split_kernel        FP64 operand -> per-row power-of-two scale, integer of
//                       <= beta bits, balanced residues mod p_j as BF16,
//                       stored K-major: S[j][row][k]            (HBM-bound)
//   crt_mma_kernel      per (output tile, modulus): C_j = A_j B_j' on tcgen05,
//                       TMA-fed 4..6-stage pipeline, FP32 accumulators in
//                       TMEM (double-buffered over moduli), epilogue reduces
//                       each exact integer sum mod p_j to one byte  (tensor)
//   reconstruct_kernel  CRT of the n residues -> exact integer -> FP64
//                       (one rounding) x 2^(scale_i + scale_j), then
//                       alpha * . + beta * C                       (integer ALU)
//
// Every spin-wait on an mbarrier has an iteration limit; on expiry the CTA
// records ST_TIMEOUT in the call's status word, stops issuing work, waits (with
// a limit) for the copies it has in flight, frees its tensor memory and exits.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "crt.h"
#include "crt_device.cuh"
#include "kernels.h"

namespace cpinv {

// ---------------------------------------------------------------------------
// host: CRT constants
// ---------------------------------------------------------------------------
namespace crt {

namespace {
// little-endian 32-bit limbs, fixed width
struct Big {
  uint32_t w[kLimbs];
};
Big big_from(uint64_t v) {
  Big b{};
  b.w[0] = (uint32_t)v;
  b.w[1] = (uint32_t)(v >> 32);
  return b;
}
Big big_mul_small(const Big& a, uint32_t m) {
  Big r{};
  uint64_t carry = 0;
  for (int i = 0; i < kLimbs; ++i) {
    uint64_t t = (uint64_t)a.w[i] * m + carry;
    r.w[i] = (uint32_t)t;
    carry = t >> 32;
  }
  return r;
}
Big big_div_small(const Big& a, uint32_t d, uint32_t* rem) {
  Big q{};
  uint64_t r = 0;
  for (int i = kLimbs - 1; i >= 0; --i) {
    uint64_t cur = (r << 32) | a.w[i];
    q.w[i] = (uint32_t)(cur / d);
    r = cur % d;
  }
  if (rem) *rem = (uint32_t)r;
  return q;
}
int big_bitlen(const Big& a) {
  for (int i = kLimbs - 1; i >= 0; --i)
    if (a.w[i]) return 32 * i + 32 - __builtin_clz(a.w[i]);
  return 0;
}
uint64_t big_shr64(const Big& a, int sh) {  // low 64 bits of a >> sh
  uint64_t r = 0;
  for (int b = 0; b < 64; ++b) {
    const int pos = sh + b;
    if (pos < 32 * kLimbs && ((a.w[pos / 32] >> (pos % 32)) & 1u)) r |= (uint64_t)1 << b;
  }
  return r;
}
}  // namespace

int moduli_for_bits(int bits) {
  double acc = 0.0;
  for (int n = 1; n <= kMaxMod; ++n) {
    acc += std::log2((double)kModuli[n - 1]);
    if (acc > (double)bits + 0.01) return n;
  }
  return -1;
}

void make_consts(int n, Consts* c) {
  std::memset(c, 0, sizeof(*c));
  c->n = n;
  Big P = big_from(1);
  for (int j = 0; j < n; ++j) P = big_mul_small(P, (uint32_t)kModuli[j]);
  std::memcpy(c->P, P.w, sizeof(P.w));
  uint32_t rem;
  Big half = big_div_small(P, 2, &rem);
  std::memcpy(c->halfP, half.w, sizeof(half.w));
  for (int j = 0; j < n; ++j) {
    const uint32_t p = (uint32_t)kModuli[j];
    Big Mj = big_div_small(P, p, &rem);
    std::memcpy(c->Mj[j], Mj.w, sizeof(Mj.w));
    uint32_t mm;
    big_div_small(Mj, p, &mm);  // Mj mod p
    uint32_t y = 0;
    for (uint32_t t = 1; t < p; ++t)
      if ((mm * t) % p == 1) {
        y = t;
        break;
      }
    for (uint32_t r = 0; r < 128; ++r) c->tab[j][r] = (uint8_t)((r * y) % p);
  }
  const int bl = big_bitlen(P);
  c->shift = bl > 58 ? bl - 58 : 0;
  const uint64_t ptop = big_shr64(P, c->shift);
  c->inv_ptop = (float)(1.0 / (double)ptop);
}

}  // namespace crt

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 128;       // rows of an output tile (TMEM lanes)
constexpr int BK = 64;        // K per pipeline stage: 64 BF16 = one 128-byte swizzle row
constexpr uint32_t kSpinLimit = 1u << 26;

// ---------------------------------------------------------------------------
// split: op(X) (rows x K, FP64) -> residues
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool nonfinite_bits(uint64_t b) { return ((b >> 52) & 0x7FF) == 0x7FF; }

// Row exponents: E[i] = max biased exponent over row i of op(X) (0 if the row
// is 0), accumulated with atomicMax into a zeroed array.
// trans = 0: row i is contiguous (X[i*ld + k]); one warp per row.
// trans = 1: row i of op(X) is column i of X; a 32-row x 8-chunk block,
//            coalesced over i, each thread scanning a slice of k.
// Batches (grid z = zo zn.nzi + zi): operand z at X + zo zX + zi zn.zXi, its
// dims read at rdev + zo zR with zi zn.zoff added to both offsets, its state
// st + zo zSt, its exponents E + z zE.
__global__ void row_expo_kernel(const double* X, int64_t ld, int trans, Dim rowsd, Dim colsd,
                                const int64_t* rdev, int32_t* E, DevState* st, int64_t zX,
                                int64_t zR, int64_t zE, int64_t zSt, ZNest zn) {
  {
    const int64_t z = blockIdx.z;
    const int64_t zo = z / zn.nzi, zi = z - zo * zn.nzi;
    X += zo * zX + zi * zn.zXi;
    rdev += zo * zR;
    E += z * zE;
    st += zo * zSt;
    rowsd.off += zi * zn.zoff;
    colsd.off += zi * zn.zoff;
  }
  const int64_t rows = eval_dim(rowsd, rdev), cols = eval_dim(colsd, rdev);
  int emax = 0, bad = 0;
  auto take = [&](uint64_t b) {
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) bad = 1;
    else if ((b << 1) != 0 && e > emax) emax = e;
  };
  int64_t i;
  if (!trans) {
    i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i < rows) {
      const uint64_t* row = reinterpret_cast<const uint64_t*>(X + i * ld);
      int64_t k = lane;
      // four loads in flight per lane
      for (; k + 96 < cols; k += 128) {
        const uint64_t b0 = row[k], b1 = row[k + 32], b2 = row[k + 64], b3 = row[k + 96];
        take(b0);
        take(b1);
        take(b2);
        take(b3);
      }
      for (; k < cols; k += 32) take(row[k]);
    }
    for (int o = 16; o; o >>= 1) {
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane != 0) return;
  } else {
    i = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    const int64_t kc = (cols + gridDim.y * 8 - 1) / (gridDim.y * 8);
    const int64_t kb = ((int64_t)blockIdx.y * 8 + (threadIdx.x >> 5)) * kc;
    const int64_t ke = kb + kc < cols ? kb + kc : cols;
    if (i < rows) {
      const uint64_t* col = reinterpret_cast<const uint64_t*>(X) + i;
      int64_t k = kb;
      for (; k + 3 < ke; k += 4) {
        const uint64_t b0 = col[k * ld], b1 = col[(k + 1) * ld], b2 = col[(k + 2) * ld],
                       b3 = col[(k + 3) * ld];
        take(b0);
        take(b1);
        take(b2);
        take(b3);
      }
      for (; k < ke; ++k) take(col[k * ld]);
    }
  }
  if (i < rows && emax > 0) atomicMax(&E[i], emax);
  if (bad) atomicOr(&st->status, ST_NONFINITE);
}

// Residue planes of the 32-row x 64-column tile (rows i0.., k0..) of op(X):
// 256 threads, each one row x eight adjacent columns, so that every modulus
// is written as one 16-byte store (eight BF16) per thread.
template <int J>
__device__ __forceinline__ void split_store8(const uint32_t (&c)[8][3], const uint32_t (&sg)[4],
                                             int n_mod, uint4* dst, size_t plane_vec) {
  if (J >= n_mod) return;
  uint32_t w[4];
#pragma unroll
  for (int h = 0; h < 4; ++h)
    w[h] = crt::residue_pair_bf16<J>(c[2 * h][0], c[2 * h][1], c[2 * h][2], c[2 * h + 1][0],
                                     c[2 * h + 1][1], c[2 * h + 1][2], sg[h]);
  dst[J * plane_vec] = make_uint4(w[0], w[1], w[2], w[3]);
}

template <int... Js>
__device__ __forceinline__ void split_store8_all(std::integer_sequence<int, Js...>,
                                                 const uint32_t (&c)[8][3], const uint32_t (&sg)[4],
                                                 int n_mod, uint4* dst, size_t plane_vec) {
  (split_store8<Js>(c, sg, n_mod, dst, plane_vec), ...);
}

// Batches (grid z = zo zn.nzi + zi): operand z at X + zo zX + zi zn.zXi, dims
// at rdev + zo zR with zi zn.zoff added to both offsets, its rows z zrow
// onwards in the planes (and in E); plane_rows = rows of one plane.
__global__ void __launch_bounds__(256) split_kernel(const double* X, int64_t ld, int trans,
                                                    Dim rowsd, Dim colsd, int64_t rows_max,
                                                    int64_t kpad, const int64_t* rdev,
                                                    const int32_t* E, int n_mod, int beta,
                                                    bf16* out, int64_t zX, int64_t zR,
                                                    int64_t zrow, int64_t plane_rows,
                                                    ZNest zn, int trim) {
  // rows padded to 66 words: 16-byte aligned, four banks apart
  __shared__ __align__(16) uint64_t tile[32][66];
  {
    const int64_t z = blockIdx.z;
    const int64_t zo = z / zn.nzi, zi = z - zo * zn.nzi;
    X += zo * zX + zi * zn.zXi;
    rdev += zo * zR;
    E += z * zrow;
    out += z * zrow * kpad;
    rowsd.off += zi * zn.zoff;
    colsd.off += zi * zn.zoff;
  }
  const int64_t rows = eval_dim(rowsd, rdev), cols = eval_dim(colsd, rdev);
  const int64_t i0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 64;
  // trim: the product reads only the K blocks inside the device-side K (and
  // always the first), so the blocks past it are not written
  if (trim && k0 > 0 && k0 >= cols) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const uint64_t* Xb = reinterpret_cast<const uint64_t*>(X);
  if (!trans) {
    for (int q = ty; q < 32; q += 8)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t i = i0 + q, k = k0 + tx + 32 * h;
        tile[q][tx + 32 * h] = (i < rows && k < cols) ? Xb[i * ld + k] : 0ull;
      }
  } else {
    for (int q = ty; q < 64; q += 8) {
      const int64_t k = k0 + q, i = i0 + tx;
      tile[tx][q] = (i < rows && k < cols) ? Xb[k * ld + i] : 0ull;
    }
  }
  __syncthreads();
  const int q = threadIdx.x >> 3, g = threadIdx.x & 7;  // row, group of eight columns
  const int64_t i = i0 + q;
  if (i >= rows_max) return;
  const int Ei = i < rows ? E[i] : 0;
  uint32_t c[8][3];
  bool ng[8];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(&tile[q][8 * g + 2 * h]);
    const uint64_t bb[2] = {v.x, v.y};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint64_t b = bb[u];
      uint64_t a = 0;
      if (!nonfinite_bits(b)) a = crt::integerize(b, Ei, beta);
      ng[2 * h + u] = (b >> 63) != 0;
      c[2 * h + u][0] = (uint32_t)(a & 0x1FFFFF);
      c[2 * h + u][1] = (uint32_t)((a >> 21) & 0x1FFFFF);
      c[2 * h + u][2] = (uint32_t)(a >> 42);
    }
  }
  uint32_t sg[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) sg[h] = (ng[2 * h] ? 0x8000u : 0u) | (ng[2 * h + 1] ? 0x80000000u : 0u);
  uint4* dst = reinterpret_cast<uint4*>(out + (size_t)i * kpad + k0 + 8 * g);
  split_store8_all(std::make_integer_sequence<int, crt::kMaxMod>{}, c, sg, n_mod, dst,
                   (size_t)plane_rows * (size_t)kpad / 8);
}

// Split precision: the row of op(X) scaled by 2^(1022 - E[i]) (|x| < 1), then
// hi = bf16(x), lo = bf16(x - hi) (through FP32), planes out[0] and out[1].
__global__ void __launch_bounds__(256) split3_kernel(const double* X, int64_t ld, int trans,
                                                     Dim rowsd, Dim colsd, int64_t rows_max,
                                                     int64_t kpad, const int64_t* rdev,
                                                     const int32_t* E, bf16* out) {
  __shared__ uint64_t tile[32][33];
  const int64_t rows = eval_dim(rowsd, rdev), cols = eval_dim(colsd, rdev);
  const int64_t i0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int q = ty; q < 32; q += 8) {
    uint64_t v = 0;
    if (!trans) {
      const int64_t i = i0 + q, k = k0 + tx;
      if (i < rows && k < cols) v = reinterpret_cast<const uint64_t*>(X)[i * ld + k];
      tile[q][tx] = v;
    } else {
      const int64_t k = k0 + q, i = i0 + tx;
      if (i < rows && k < cols) v = reinterpret_cast<const uint64_t*>(X)[k * ld + i];
      tile[tx][q] = v;
    }
  }
  __syncthreads();
  const size_t plane = (size_t)rows_max * (size_t)kpad;
  for (int q = ty; q < 32; q += 8) {
    const int64_t i = i0 + q, k = k0 + tx;
    if (i >= rows_max || k >= kpad) continue;
    const uint64_t b = tile[q][tx];
    float xf = 0.0f;
    if (i < rows && k < cols && !nonfinite_bits(b) && E[i] > 0 && (b << 1) != 0) {
      const int ex = (int)((b >> 52) & 0x7FF);
      const int ne = ex - (E[i] - 1022);  // biased exponent of x * 2^(1022 - E[i])
      if (ex != 0 && ne > 0) {
        const uint64_t sb = (b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)ne << 52);
        xf = (float)__longlong_as_double((long long)sb);
      }
    }
    const bf16 hi = __float2bfloat16_rn(xf);
    const bf16 lo = __float2bfloat16_rn(xf - __bfloat162float(hi));
    out[(size_t)i * kpad + k] = hi;
    out[plane + (size_t)i * kpad + k] = lo;
  }
}

// ---------------------------------------------------------------------------
// tcgen05 / TMA / mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false on timeout (or if another role already gave up)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 1023u) == 1023u && *abort) return false;
    if (it > 4096) __nanosleep(64);
  }
  *abort = 1;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused, K-major SW128)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                     // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                     // layout: 128-byte swizzle
  return d;
}

template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc_bf16() {
  return (1u << 4)                 // D: FP32
         | (1u << 7)               // A: BF16
         | (1u << 10)              // B: BF16
         | ((uint32_t)(BN >> 3) << 17)
         | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// the tensor-core kernel
// ---------------------------------------------------------------------------

struct MmaParams {
  Dim M, N;                 // output size (may depend on the device rank)
  int32_t a_row0, b_row0;   // first residue row of op(A) / of the N x K view of op(B)
  const int64_t* rdev;
  int32_t nk;               // K / BK (K padded)
  int32_t kdev;             // 1: only the K blocks inside Kd (a device-side K) are summed
  Dim Kd;
  int32_t n_mod;
  int32_t tiles_m, tiles_n;  // output tiles (BM x BN) covering M.max x N.max
  int32_t tiles;             // tiles in the enumeration (the lower ones only when lower)
  int32_t pad_t;
  int32_t lower;            // skip tiles strictly above the diagonal
  int32_t blk;              // > 0: block-diagonal output of blocks blk x blk (batched Gram
                            // matrices); tiles and lower refer to one block, R holds
                            // [n_mod][Mpad][blk] (the block's own columns)
  int32_t tiles_blk;        // tiles per block
  int32_t bdims;            // block mode: block z = zo bnzi + zi has rows < bM and columns
  int32_t bnzi;             // < bN (zi bzoff added to both offsets, read at rdev + zo bzR);
  int64_t bzoff, bzR;       // the tiles past them are skipped
  Dim bM, bN;
  uint8_t* R;               // residues [n_mod][Mpad][Npad]
  int64_t Mpad, Npad;
  int32_t* status;          // DevState::status
  // split (hi/lo) variant: FP64 output written by the epilogue
  double* C;
  int64_t ldc;
  const int32_t* EA;
  const int32_t* EB;
  double alpha, beta;
};

// alpha x + beta c, with the alpha == 1 and beta == 0 tests on the bit
// patterns (integer compares: an FP64 compare takes a slot of the narrow
// FP64 pipe, and these run once per output); out of line, called only when
// plain_store() is false, so the common path executes no FP64 instruction.
__device__ __forceinline__ bool plain_store(double alpha, double beta) {
  return __double_as_longlong(alpha) == 0x3FF0000000000000ll &&
         ((uint64_t)__double_as_longlong(beta) << 1) == 0;
}
__device__ __noinline__ double scale_add(double x, double alpha, double beta, const double* c) {
  if (__double_as_longlong(alpha) != 0x3FF0000000000000ll) x *= alpha;
  if (((uint64_t)__double_as_longlong(beta) << 1) != 0) x = fma(beta, *c, x);
  return x;
}

// FP32 value * 2^s as FP64 with integer operations (exact: FP64 holds every
// FP32 value); the FP64 unit only for out-of-range exponents and subnormals.
__device__ __forceinline__ double f32_scaled_to_f64(uint32_t u, int s) {
  const uint32_t e = (u >> 23) & 0xFFu;
  if ((u << 1) == 0) return (u >> 31) ? -0.0 : 0.0;
  const int be = (int)e - 127 + 1023 + s;
  if (e == 0 || e == 0xFFu || be <= 0 || be >= 2047)
    return ldexp((double)__uint_as_float(u), s);
  const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)be << 52) |
                        ((uint64_t)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

template <int BN, int STAGES, int PL>
struct __align__(1024) MmaSmem {
  bf16 A[STAGES][PL][BM * BK];
  bf16 B[STAGES][PL][BN * BK];
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t accfull[2];
  uint64_t accempty[2];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

// S3 = false: residue products, one job per modulus (crt.h).
// S3 = true: split precision, one job; planes 0/1 hold the hi/lo BF16 parts of
// the scaled operands and each K step accumulates hi*hi + hi*lo + lo*hi in
// FP32; the epilogue writes alpha * 2^(e_i + e_j) acc + beta C in FP64.
template <int BN, int STAGES, bool S3>
__global__ void __launch_bounds__(192, 1)
    crt_mma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   MmaParams p) {
  constexpr int PL = S3 ? 2 : 1;
  extern __shared__ uint8_t smem_raw[];
  MmaSmem<BN, STAGES, PL>& sm = *reinterpret_cast<MmaSmem<BN, STAGES, PL>*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int64_t M = eval_dim(p.M, p.rdev), N = eval_dim(p.N, p.rdev);
  // Jobs are the (modulus, tile) pairs, modulus-major; CTA c runs jobs c,
  // c + G, c + 2G, ... (G CTAs), so every CTA gets the same number of jobs
  // to within one and the CTAs running at the same time work on
  // neighbouring tiles of the same modulus (their operand tiles are shared
  // in L2).  Jobs on tiles outside the output (a device-side size below its
  // maximum) are skipped by every role alike.
  const int64_t J = (int64_t)p.tiles * p.n_mod;
  const int64_t G = gridDim.x;
  const int njobs = (int)((J - (int64_t)blockIdx.x + G - 1) / G);
  if (njobs <= 0) return;
  // job -> (m0, n0, modulus); false when the job has no output
  auto job = [&](int jj, int64_t& m0, int64_t& n0, int& j) -> bool {
    const int64_t q = (int64_t)blockIdx.x + (int64_t)jj * G;
    j = (int)(q / p.tiles);
    int t = (int)(q - (int64_t)j * p.tiles);
    int64_t base = 0;  // block-diagonal mode: first row and column of the block
    int64_t bmv = BM * (int64_t)p.tiles_m, bnv = BN * (int64_t)p.tiles_n;  // block's extent
    if (p.blk) {
      const int zb = t / p.tiles_blk;
      t -= zb * p.tiles_blk;
      base = (int64_t)zb * p.blk;
      if (p.bdims) {
        const int zo = zb / p.bnzi, zi = zb - zo * p.bnzi;
        Dim dm = p.bM, dn = p.bN;
        dm.off += zi * p.bzoff;
        dn.off += zi * p.bzoff;
        bmv = eval_dim(dm, p.rdev + zo * p.bzR);
        bnv = eval_dim(dn, p.rdev + zo * p.bzR);
      }
    }
    int ty, tx;
    if (!p.lower) {
      ty = t / p.tiles_n;
      tx = t - ty * p.tiles_n;
    } else {  // row ty holds the tiles tx with tx BN <= ty BM + BM - 1
      int rem = t;
      ty = 0;
      for (;;) {
        int cnt = (ty * BM + BM - 1) / BN + 1;
        cnt = cnt < p.tiles_n ? cnt : p.tiles_n;
        if (rem < cnt || ty + 1 >= p.tiles_m) break;
        rem -= cnt;
        ++ty;
      }
      tx = rem;
    }
    m0 = (int64_t)ty * BM;
    n0 = (int64_t)tx * BN;
    const bool upper = p.lower && n0 > m0 + BM - 1;
    const bool inside = m0 < bmv && n0 < bnv;
    m0 += base;
    n0 += base;
    return m0 < M && n0 < N && !upper && inside;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&sm.accfull[a], 1);
      mbar_init(&sm.accempty[a], 4);
    }
    mbar_init(&sm.done, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sm.tmem_base)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort = &sm.abort;
  constexpr uint32_t kStageBytes = PL * (BM + BN) * BK * sizeof(bf16);
  // K blocks past a device-side K hold zero residues: not summed (at least
  // one block, so that every accumulator is written)
  int nk = p.nk;
  if (p.kdev) {
    const int64_t kv = (eval_dim(p.Kd, p.rdev) + BK - 1) / BK;
    nk = kv < 1 ? 1 : (kv < nk ? (int)kv : nk);
  }

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      for (int jj = 0; jj < njobs && !*abort; ++jj) {
        int64_t m0, n0;
        int j;
        if (!job(jj, m0, n0, j)) continue;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait(&sm.empty[s], ph ^ 1u, abort)) break;
          mbar_expect_tx(&sm.full[s], kStageBytes);
#pragma unroll
          for (int pl = 0; pl < PL; ++pl) {
            const int z = S3 ? pl : j;
            tma_load_3d(sm.A[s][pl], &tmA, &sm.full[s], kb * BK, p.a_row0 + (int)m0, z);
            tma_load_3d(sm.B[s][pl], &tmB, &sm.full[s], kb * BK, p.b_row0 + (int)n0, z);
          }
        }
      }
      // drain: every issued stage must have landed before the CTA exits
      const uint32_t issued = it;
      for (uint32_t q = issued > STAGES ? issued - STAGES : 0; q < issued; ++q) {
        const int s = (int)(q % STAGES);
        for (uint32_t t = 0; t < kSpinLimit && !mbar_try(&sm.full[s], (q / STAGES) & 1u); ++t) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16<BN>();
      uint32_t it = 0;
      int na = 0;  // active jobs so far (the accumulator sequence)
      for (int jj = 0; jj < njobs && !*abort; ++jj) {
        int64_t m0, n0;
        int j;
        if (!job(jj, m0, n0, j)) continue;
        const int acc = na & 1;
        if (!mbar_wait(&sm.accempty[acc], ((na >> 1) & 1u) ^ 1u, abort)) break;
        ++na;
        tc_fence_after();
        const uint32_t dtm = tmem + (uint32_t)(acc * BN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (!mbar_wait(&sm.full[s], (it / STAGES) & 1u, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sm.A[s][0]), b0 = smem_u32(sm.B[s][0]);
#pragma unroll
          for (int ks = 0; ks < BK / 16; ++ks) {
            umma_bf16(dtm, umma_desc_sw128(a0 + ks * 32), umma_desc_sw128(b0 + ks * 32), idesc,
                      (kb | ks) != 0);
            if constexpr (S3) {
              const uint32_t a1 = smem_u32(sm.A[s][PL - 1]), b1 = smem_u32(sm.B[s][PL - 1]);
              umma_bf16(dtm, umma_desc_sw128(a0 + ks * 32), umma_desc_sw128(b1 + ks * 32), idesc, 1);
              umma_bf16(dtm, umma_desc_sw128(a1 + ks * 32), umma_desc_sw128(b0 + ks * 32), idesc, 1);
            }
          }
          umma_commit(&sm.empty[s]);  // stage reusable once these MMAs are done
        }
        if (!ok) break;
        umma_commit(&sm.accfull[acc]);
      }
      // every MMA issued by this thread has finished once `done` completes
      umma_commit(&sm.done);
      for (uint32_t t = 0; t < kSpinLimit && !mbar_try(&sm.done, 0); ++t) {
      }
    }
  } else {
    // ---------------- epilogue: 4 warps, warp w reads TMEM lanes 32*(w%4).. ----------------
    const int q = warp & 3;
    int na = 0;
    for (int jj = 0; jj < njobs; ++jj) {
      int64_t m0, n0;
      int j;
      if (!job(jj, m0, n0, j)) continue;
      const int acc = na & 1;
      if (!mbar_wait(&sm.accfull[acc], (na >> 1) & 1u, abort)) break;
      ++na;
      const int64_t row = m0 + q * 32 + lane;
      tc_fence_after();
      if constexpr (S3) {
        const int64_t Mv = M, Nv = N;
        const bool rowok = row < Mv;
        const int sr = rowok ? p.EA[row] - 1022 : 0;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c), v);
          if (!rowok) continue;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int64_t col = n0 + c + e;
            if (col >= Nv || (p.lower && col > row)) continue;
            double d = f32_scaled_to_f64(v[e], sr + p.EB[col] - 1022);
            double* cp = p.C + row * p.ldc + col;
            if (!plain_store(p.alpha, p.beta)) d = scale_add(d, p.alpha, p.beta, cp);
            *cp = d;
          }
        }
      } else {
        int pj = 0;
  #pragma unroll
        for (int t = 0; t < crt::kMaxMod; ++t)
          if (t == j) pj = crt::modulus(t);
        const float pfl = (float)pj, inv = 1.0f / (float)pj;
        // block-diagonal mode: the block's own column n0 - base
        const int64_t nc = p.blk ? n0 - (m0 / p.blk) * p.blk : n0;
        uint8_t* out = p.R + ((size_t)j * p.Mpad + row) * p.Npad + nc;
  #pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c), v);
          uint32_t packed[8];
  #pragma unroll
          for (int e = 0; e < 32; ++e) {
            // exact integer |x| <= 2^24: x mod p in [0, p)
            const float x = __uint_as_float(v[e]);
            float qf = floorf(x * inv);
            float r = fmaf(-qf, pfl, x);
            if (r < 0.f) r += pfl;
            if (r >= pfl) r -= pfl;
            const uint32_t rb = __float_as_uint(r + 8388608.0f) & 0xFFu;  // 2^23 trick
            if ((e & 3) == 0) packed[e >> 2] = 0;
            packed[e >> 2] |= rb << (8 * (e & 3));
          }
          uint4* dst = reinterpret_cast<uint4*>(out + c);
          dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.accempty[acc]);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
  if (threadIdx.x == 0 && sm.abort) atomicOr(p.status, ST_TIMEOUT);
}

// ---------------------------------------------------------------------------
// reconstruction
// ---------------------------------------------------------------------------

struct ReconParams {
  const uint8_t* R;
  int64_t Mpad, Npad;
  Dim M, N;
  const int64_t* rdev;
  const int32_t* EA;  // biased exponent maxima of the rows of op(A)
  const int32_t* EB;  // ... of the columns of op(B)
  int32_t betaA, betaB;
  double alpha, beta;
  double* C;
  int64_t ldc;
  int32_t lower;
  int32_t blk;  // > 0: block-diagonal output (reconstruct_words_kernel only): row i
                // belongs to block z = i / blk, its columns j are the block's own
                // (EB[z blk + j]), lower is within the block; the row goes to
                // C + z zC + (i - z blk) ldc
  int32_t bdims;  // block mode, z = zo bnzi + zi: block z keeps its rows il < bM and
                  // columns j < bN (zi zoff added to their offsets, read at rdev +
                  // zo bzR) and goes to C + zo zCo + zi zC + il ldc
  int32_t bnzi;
  int64_t zC, zCo, zoff, bzR;
  Dim bM, bN;
};

// CRT constants of every moduli count, in device memory (uploaded once per
// device): blocks read them with coalesced loads.
__device__ crt::Consts g_crt_consts[crt::kMaxMod + 1];

// Two adjacent columns per thread: the residue bytes of a modulus come in one
// 16-bit load and each multiplier P/p_j is read once for both sums.
constexpr int kRecW = 2;

__global__ void __launch_bounds__(256, 2) reconstruct_kernel(ReconParams p, int n_mod) {
  const crt::Consts& c = g_crt_consts[n_mod];
  __shared__ crt::CrtShared sh;
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&c.tab[0][0]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sh.tab[0][0]);
    for (int e = threadIdx.x; e < n_mod * 32; e += blockDim.x) dst[e] = src[e];
    for (int e = threadIdx.x; e < n_mod * crt::kLimbs; e += blockDim.x)
      sh.Mj[e / crt::kLimbs][e % crt::kLimbs] = c.Mj[e / crt::kLimbs][e % crt::kLimbs];
  }
  __syncthreads();
  if (threadIdx.x < crt::kLimbs) {
    sh.P[threadIdx.x] = c.P[threadIdx.x];
    sh.halfP[threadIdx.x] = c.halfP[threadIdx.x];
  }
  __syncthreads();
  const int n = n_mod;
  const int shift = c.shift;
  const float inv_ptop = c.inv_ptop;
  const int64_t M = eval_dim(p.M, p.rdev), N = eval_dim(p.N, p.rdev);
  const int64_t NG = (N + kRecW - 1) / kRecW;  // column groups
  const int64_t total = M * NG;
  const size_t plane = (size_t)p.Mpad * (size_t)p.Npad;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / NG, j0 = (idx - i * NG) * kRecW;
    if (p.lower && j0 > i) continue;
    const uint16_t* r = reinterpret_cast<const uint16_t*>(p.R + i * p.Npad + j0);
    uint64_t acc[kRecW][crt::kLimbs];
#pragma unroll
    for (int e = 0; e < kRecW; ++e)
#pragma unroll
      for (int l = 0; l < crt::kLimbs; ++l) acc[e][l] = 0;
    // residues in groups of eight loads in flight, then their sums
#pragma unroll
    for (int m0 = 0; m0 < crt::kMaxMod; m0 += 8) {
      uint32_t rv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) rv[q] = (m0 + q) < n ? r[(m0 + q) * (plane / kRecW)] : 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int m = m0 + q;
        if (m < n) {
          uint32_t mj[crt::kLimbs];
#pragma unroll
          for (int l = 0; l < crt::kLimbs; ++l) mj[l] = sh.Mj[m][l];
#pragma unroll
          for (int e = 0; e < kRecW; ++e) {
            const uint32_t t = sh.tab[m][(rv[q] >> (8 * e)) & 0xFFu];
#pragma unroll
            for (int l = 0; l < crt::kLimbs; ++l) acc[e][l] += (uint64_t)t * mj[l];
          }
        }
      }
    }
    const int sa = p.EA[i] - 1022 - p.betaA;
#pragma unroll
    for (int e = 0; e < kRecW; ++e) {
      const int64_t j = j0 + e;
      if (j >= N || (p.lower && j > i)) continue;
      uint32_t S[crt::kLimbs];
      uint64_t carry = 0;
#pragma unroll
      for (int l = 0; l < crt::kLimbs; ++l) {
        const uint64_t v = acc[e][l] + carry;
        S[l] = (uint32_t)v;
        carry = v >> 32;
      }
      double v = crt::crt_finish(S, sh.P, sh.halfP, shift, inv_ptop, sa + p.EB[j] - 1022 - p.betaB);
      double* cp = p.C + i * p.ldc + j;
      if (!plain_store(p.alpha, p.beta)) v = scale_add(v, p.alpha, p.beta, cp);
      *cp = v;
    }
  }
}

// Reconstruction on 64-bit words, for n_mod <= 22 (P < 2^143).  NL = 4
// limbs of 32 bits hold every multiplier P / p_j when P < 2^128 (n_mod <=
// 19: the FP64-accurate products of the chain), NL = 5 otherwise (the
// Gram's and the factorisation's wider products).  The CRT sum S (< n P)
// lives in three 64-bit words; the reduction mod P uses a quotient estimate
// from FP32, the centring and the rounding work word-wise.  Four adjacent
// columns per thread (one 32-bit load per modulus), LW threads per row:
// eight rows x 128 columns per block, or (LW = 8, outputs of at most 32
// columns) 32 rows x 32 columns.
constexpr int kRecWordsMaxMod = 22;
constexpr int kRecWords4MaxMod = 19;
static_assert(kRecWordsMaxMod == kRecBlockMaxMod, "block-diagonal reconstruction limit");
constexpr int kRecWRows = 8, kRecWCols = 128;
struct __align__(16) RecWShared {
  uint32_t Mj[crt::kMaxMod][8];  // P / p_j, limbs 0..4, padded
  uint8_t tab[crt::kMaxMod][128];
};

// +-mant * 2^e outside the normal exponent range (the FP64 unit rounds the
// underflow); out of line, so that the common path never executes it.
__device__ __noinline__ double scaled_out_of_range(bool neg, uint64_t mant, int e) {
  const double d = ldexp((double)mant, e);
  return neg ? -d : d;
}

// Correctly rounded (m2:m1:m0) * 2^scale with sign, by integer operations.
__device__ __forceinline__ double u192_to_double(bool neg, uint64_t m2, uint64_t m1, uint64_t m0,
                                                 int scale) {
  int top;
  uint64_t t;  // the 64 bits from the leading one down
  bool sticky;
  if (m2) {
    const int lz = __clzll((long long)m2);
    top = 191 - lz;
    t = lz ? (m2 << lz) | (m1 >> (64 - lz)) : m2;
    sticky = (lz ? (m1 << lz) != 0 : m1 != 0) || m0 != 0;
  } else if (m1) {
    const int lz = __clzll((long long)m1);
    top = 127 - lz;
    t = lz ? (m1 << lz) | (m0 >> (64 - lz)) : m1;
    sticky = lz ? (m0 << lz) != 0 : m0 != 0;
  } else if (m0) {
    const int lz = __clzll((long long)m0);
    top = 63 - lz;
    t = m0 << lz;
    sticky = false;
  } else {
    return neg ? -0.0 : 0.0;
  }
  uint64_t mant = t >> 11;
  const uint64_t rem = t & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (sticky || (mant & 1ull)))) ++mant;
  int e = top;  // value = mant * 2^(top - 52)
  if (mant >> 53) {
    mant >>= 1;
    ++e;
  }
  const int biased = e + scale + 1023;
  if (biased <= 0 || biased >= 2047) return scaled_out_of_range(neg, mant, e - 52 + scale);
  return __longlong_as_double(
      (long long)(((uint64_t)neg << 63) | ((uint64_t)biased << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// The low 64 bits of (s2:s1:s0) >> sh, 0 <= sh < 192.
__device__ __forceinline__ uint64_t shr192(uint64_t s2, uint64_t s1, uint64_t s0, int sh) {
  if (sh >= 128) return s2 >> (sh - 128);
  if (sh >= 64) return sh == 64 ? s1 : (s1 >> (sh - 64)) | (s2 << (128 - sh));
  return sh == 0 ? s0 : (s0 >> sh) | (s1 << (64 - sh));
}

// (x2:x1:x0) += (y2:y1:y0) or -= , modulo 2^192
__device__ __forceinline__ void add192(uint64_t& x2, uint64_t& x1, uint64_t& x0, uint64_t y2,
                                       uint64_t y1, uint64_t y0) {
  x0 += y0;
  const uint64_t c0 = x0 < y0;
  const uint64_t t1 = x1 + y1;
  const uint64_t c1 = t1 < x1;
  x1 = t1 + c0;
  x2 += y2 + c1 + (x1 < c0 ? 1u : 0u);
}
__device__ __forceinline__ void sub192(uint64_t& x2, uint64_t& x1, uint64_t& x0, uint64_t y2,
                                       uint64_t y1, uint64_t y0) {
  const uint64_t b0 = x0 < y0;
  x0 -= y0;
  const uint64_t b1 = (x1 < y1) || (x1 == y1 && b0);
  x1 = x1 - y1 - b0;
  x2 = x2 - y2 - b1;
}
__device__ __forceinline__ bool gt192(uint64_t x2, uint64_t x1, uint64_t x0, uint64_t y2,
                                      uint64_t y1, uint64_t y0) {
  return x2 != y2 ? x2 > y2 : (x1 != y1 ? x1 > y1 : x0 > y0);
}

template <int NL, int LW>
__global__ void __launch_bounds__(256) reconstruct_words_kernel(ReconParams p, int n_mod) {
  const crt::Consts& c = g_crt_consts[n_mod];
  __shared__ RecWShared sh;
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&c.tab[0][0]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sh.tab[0][0]);
    for (int e = threadIdx.x; e < n_mod * 32; e += blockDim.x) dst[e] = src[e];
    for (int e = threadIdx.x; e < n_mod * 8; e += blockDim.x)
      sh.Mj[e >> 3][e & 7] = (e & 7) < crt::kLimbs ? c.Mj[e >> 3][e & 7] : 0u;
  }
  __syncthreads();
  const uint64_t P0 = c.P[0] | ((uint64_t)c.P[1] << 32), P1 = c.P[2] | ((uint64_t)c.P[3] << 32);
  const uint64_t P2 = c.P[4];
  const uint64_t H0 = c.halfP[0] | ((uint64_t)c.halfP[1] << 32),
                 H1 = c.halfP[2] | ((uint64_t)c.halfP[3] << 32);
  const uint64_t H2 = c.halfP[4];
  // quotient estimate floor(S / P) from the 24 leading bits of P: S >> qs
  // is below n 2^24 < 2^29, so FP32 holds it with a relative error of 2^-24
  const int pbits = P2   ? 192 - __clzll((long long)P2)
                    : P1 ? 128 - __clzll((long long)P1)
                         : 64 - __clzll((long long)P0);
  const int qs = pbits > 24 ? pbits - 24 : 0;
  const float inv_ptop = 1.0f / (float)(uint32_t)shr192(P2, P1, P0, qs);

  const int64_t M = eval_dim(p.M, p.rdev), N = eval_dim(p.N, p.rdev);
  const int64_t i = (int64_t)blockIdx.y * (256 / LW) + (threadIdx.x / LW);
  const int64_t j0 = (int64_t)blockIdx.x * (4 * LW) + 4 * (threadIdx.x % LW);
  const int64_t il = p.blk ? i % p.blk : i;       // row within its block
  const int64_t zb = p.blk ? i / p.blk : 0;
  const int32_t* EB = p.blk ? p.EB + (i - il) : p.EB;
  int64_t Nv = N;
  bool row_ok = i < M;
  int64_t coff = zb * p.zC;
  if (p.bdims) {
    const int64_t zo = zb / p.bnzi, zi = zb - zo * p.bnzi;
    Dim bm = p.bM, bn = p.bN;
    bm.off += zi * p.zoff;
    bn.off += zi * p.zoff;
    row_ok = row_ok && il < eval_dim(bm, p.rdev + zo * p.bzR);
    Nv = eval_dim(bn, p.rdev + zo * p.bzR);
    coff = zo * p.zCo + zi * p.zC;
  }
  if (!row_ok || j0 >= Nv || (p.lower && j0 > il)) return;
  double* crow = p.C + (p.blk ? coff + il * p.ldc : i * p.ldc);
  const size_t plane = (size_t)p.Mpad * (size_t)p.Npad;
  const uint32_t* r = reinterpret_cast<const uint32_t*>(p.R + i * p.Npad + j0);
  uint64_t acc[4][NL];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int l = 0; l < NL; ++l) acc[e][l] = 0;
  // residues in groups of seven loads in flight, then their sums
#pragma unroll
  for (int m0 = 0; m0 < kRecWordsMaxMod; m0 += 7) {
    uint32_t rv[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) rv[q] = (m0 + q) < n_mod ? r[(size_t)(m0 + q) * (plane / 4)] : 0u;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const int m = m0 + q;
      if (m < n_mod) {
        const uint4 mj = *reinterpret_cast<const uint4*>(&sh.Mj[m][0]);
        const uint32_t mj4 = NL > 4 ? sh.Mj[m][4] : 0u;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint64_t t = sh.tab[m][(rv[q] >> (8 * e)) & 0xFFu];
          acc[e][0] += t * mj.x;
          acc[e][1] += t * mj.y;
          acc[e][2] += t * mj.z;
          acc[e][3] += t * mj.w;
          if (NL > 4) acc[e][NL - 1] += t * mj4;
        }
      }
    }
  }
  const int sa = p.EA[i] - 1022 - p.betaA;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t j = j0 + e;
    if (j >= Nv || (p.lower && j > il)) continue;
    // S = sum_j t_j P/p_j (< n P) as (s2:s1:s0)
    uint32_t Sl[6];
    uint64_t carry = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const uint64_t v = acc[e][l] + carry;
      Sl[l] = (uint32_t)v;
      carry = v >> 32;
    }
    Sl[NL] = (uint32_t)carry;
    if (NL == 4) Sl[5] = 0;
    const uint64_t s0 = Sl[0] | ((uint64_t)Sl[1] << 32), s1 = Sl[2] | ((uint64_t)Sl[3] << 32);
    const uint64_t s2 = Sl[4] | ((uint64_t)Sl[5] << 32);
    // X = S - q P, then into [0, P) (the estimate is off by at most one)
    // (through a 32-bit integer: a float to 64-bit integer conversion would
    // run on the FP64 pipe)
    const uint64_t q = (uint32_t)floorf((float)(uint32_t)shr192(s2, s1, s0, qs) * inv_ptop);
    const uint64_t qp0 = q * P0;
    const uint64_t c0 = __umul64hi(q, P0);
    const uint64_t qp1 = q * P1 + c0;
    const uint64_t qp2 = __umul64hi(q, P1) + (qp1 < c0 ? 1u : 0u) + q * P2;
    uint64_t x0 = s0, x1 = s1, x2 = s2;
    sub192(x2, x1, x0, qp2, qp1, qp0);
    if ((int64_t)x2 < 0) add192(x2, x1, x0, P2, P1, P0);
    else if (!gt192(P2, P1, P0, x2, x1, x0)) sub192(x2, x1, x0, P2, P1, P0);  // X >= P
    // centre into (-P/2, P/2]
    const bool neg = gt192(x2, x1, x0, H2, H1, H0);
    if (neg) {
      uint64_t m2 = P2, m1 = P1, m0 = P0;
      sub192(m2, m1, m0, x2, x1, x0);
      x2 = m2;
      x1 = m1;
      x0 = m0;
    }
    double v = u192_to_double(neg, NL > 4 ? x2 : 0, x1, x0, sa + EB[j] - 1022 - p.betaB);
    double* cp = crow + j;
    if (!plain_store(p.alpha, p.beta)) v = scale_add(v, p.alpha, p.beta, cp);
    *cp = v;
  }
}

// The same reconstruction for small outputs (the panel updates of the
// factorisation): four lanes share one output, each summing every fourth
// modulus, and the partial sums meet by shuffles, so an output's latency
// chain is a quarter of the moduli long and four times as many threads run.
constexpr int kRecLanes = 4;

__global__ void __launch_bounds__(256) reconstruct_split_kernel(ReconParams p, int n_mod) {
  const crt::Consts& c = g_crt_consts[n_mod];
  __shared__ crt::CrtShared sh;
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&c.tab[0][0]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sh.tab[0][0]);
    for (int e = threadIdx.x; e < n_mod * 32; e += blockDim.x) dst[e] = src[e];
    for (int e = threadIdx.x; e < n_mod * crt::kLimbs; e += blockDim.x)
      sh.Mj[e / crt::kLimbs][e % crt::kLimbs] = c.Mj[e / crt::kLimbs][e % crt::kLimbs];
  }
  if (threadIdx.x < crt::kLimbs) {
    sh.P[threadIdx.x] = c.P[threadIdx.x];
    sh.halfP[threadIdx.x] = c.halfP[threadIdx.x];
  }
  __syncthreads();
  const int n = n_mod;
  const int64_t M = eval_dim(p.M, p.rdev), N = eval_dim(p.N, p.rdev);
  const int64_t total = M * N * kRecLanes;
  const size_t plane = (size_t)p.Mpad * (size_t)p.Npad;
  const int lane = threadIdx.x & 31, g = lane & (kRecLanes - 1);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform trip count: every lane reaches the shuffles
  for (int64_t wb = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); wb < total;
       wb += stride) {
    const int64_t idx = wb + lane;
    const int64_t o = idx / kRecLanes;
    const int64_t i = o / (N > 0 ? N : 1), j = o - i * N;
    const bool active = idx < total && !(p.lower && j > i);
    uint64_t acc[crt::kLimbs];
#pragma unroll
    for (int l = 0; l < crt::kLimbs; ++l) acc[l] = 0;
    if (active) {
      const uint8_t* r = p.R + i * p.Npad + j;
#pragma unroll
      for (int t = 0; t < crt::kMaxMod / kRecLanes; ++t) {
        const int m = g + kRecLanes * t;
        if (m < n) {
          const uint32_t tv = sh.tab[m][r[(size_t)m * plane]];
#pragma unroll
          for (int l = 0; l < crt::kLimbs; ++l) acc[l] += (uint64_t)tv * sh.Mj[m][l];
        }
      }
    }
#pragma unroll
    for (int off = 1; off < kRecLanes; off <<= 1)
#pragma unroll
      for (int l = 0; l < crt::kLimbs; ++l)
        acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], off);
    if (!active || g != 0) continue;
    uint32_t S[crt::kLimbs];
    uint64_t carry = 0;
#pragma unroll
    for (int l = 0; l < crt::kLimbs; ++l) {
      const uint64_t v = acc[l] + carry;
      S[l] = (uint32_t)v;
      carry = v >> 32;
    }
    double v = crt::crt_finish(S, sh.P, sh.halfP, c.shift, c.inv_ptop,
                          p.EA[i] - 1022 - p.betaA + p.EB[j] - 1022 - p.betaB);
    double* cp = p.C + i * p.ldc + j;
    if (!plain_store(p.alpha, p.beta)) v = scale_add(v, p.alpha, p.beta, cp);
    *cp = v;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

bool make_map(CUtensorMap* map, const bf16* base, int64_t kpad, int64_t rows, int n_mod,
              int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)n_mod};
  cuuint64_t strides[2] = {(cuuint64_t)(kpad * sizeof(bf16)),
                           (cuuint64_t)(kpad * rows * sizeof(bf16))};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The grid: `wave` CTAs (one per SM, or fewer to leave SMs to concurrent
// work) taking the (modulus, tile) jobs in turn; fewer when there are fewer
// jobs.
template <int BN, int STAGES, bool S3>
cudaError_t launch_mma(const CUtensorMap& ta, CUtensorMap const& tb, MmaParams& mp,
                       int64_t Mmax, int64_t Nmax, int64_t wave, cudaStream_t s) {
  // block-diagonal mode: the tiles of one blk x blk block (of its kept rows
  // and columns when they are bounded), times the blocks
  int64_t bm = mp.blk ? mp.blk : Mmax, bn = mp.blk ? mp.blk : Nmax;
  if (mp.blk && mp.bdims) {
    bm = std::min<int64_t>(bm, mp.bM.max);
    bn = std::min<int64_t>(bn, mp.bN.max);
    if (bm < 1 || bn < 1) return cudaSuccess;
  }
  mp.tiles_m = (int32_t)((bm + BM - 1) / BM);
  mp.tiles_n = (int32_t)((bn + BN - 1) / BN);
  int64_t tiles = 0;
  if (!mp.lower) {
    tiles = (int64_t)mp.tiles_m * mp.tiles_n;
  } else {
    for (int ty = 0; ty < mp.tiles_m; ++ty) {
      const int64_t cnt = ((int64_t)ty * BM + BM - 1) / BN + 1;
      tiles += cnt < mp.tiles_n ? cnt : mp.tiles_n;
    }
  }
  if (mp.blk) {
    if (mp.blk % BM || mp.blk % BN || Mmax % mp.blk || Nmax != Mmax) return cudaErrorInvalidValue;
    mp.tiles_blk = (int32_t)tiles;
    tiles *= Mmax / mp.blk;
  }
  if (tiles > INT32_MAX) return cudaErrorInvalidValue;
  mp.tiles = (int32_t)tiles;
  const int64_t jobs = tiles * mp.n_mod;
  const int64_t ctas = jobs < wave ? jobs : wave;
  if (ctas <= 0) return cudaSuccess;
  const size_t smem = sizeof(MmaSmem<BN, STAGES, S3 ? 2 : 1>) + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(crt_mma_kernel<BN, STAGES, S3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // largest carveout: room beside this CTA for kernels on other streams
    e = cudaFuncSetAttribute(crt_mma_kernel<BN, STAGES, S3>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  crt_mma_kernel<BN, STAGES, S3><<<dim3((unsigned)ctas), 192, smem, s>>>(ta, tb, mp);
  return cudaGetLastError();
}

inline unsigned grid1d(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

// Moduli needed so that 2 K 2^(betaA + betaB) < prod p_j (one bit of margin).
int crt_moduli_for(int64_t Kmax, int betaA, int betaB) {
  const int bits = 1 + (int)std::ceil(std::log2((double)(Kmax > 1 ? Kmax : 2))) + betaA + betaB + 1;
  return crt::moduli_for_bits(bits);
}

int crt_block_k() { return BK; }
int crt_block_m() { return BM; }

// Workspace needed by one exact product (see launch_crt_gemm).
size_t crt_workspace_bytes(int64_t Mmax, int64_t Nmax, int64_t Kmax, int n_mod, bool same_operand) {
  const int64_t kpad = round_up(Kmax > 0 ? Kmax : 1, BK);
  const int64_t mpad = round_up(Mmax > 0 ? Mmax : 1, BM);
  const int64_t npad = round_up(Nmax > 0 ? Nmax : 1, 256);
  size_t b = 0;
  auto add = [&](size_t x) { b = (b + 1023) / 1024 * 1024 + x; };
  add(sizeof(bf16) * (size_t)n_mod * (size_t)mpad * (size_t)kpad);  // A slices
  if (!same_operand) add(sizeof(bf16) * (size_t)n_mod * (size_t)npad * (size_t)kpad);
  add((size_t)n_mod * (size_t)mpad * (size_t)npad);  // residues
  add(sizeof(int32_t) * (size_t)(mpad + npad));      // exponents
  return b + 1024;
}

cudaError_t crt_row_exponents(const double* X, int64_t ld, int tview, Dim rows, Dim K,
                              const int64_t* rdev, int64_t rows_max, int32_t* E, DevState* st,
                              cudaStream_t s, KernelTimer* timer) {
  return crt_row_exponents_batched(X, ld, tview, rows, K, rdev, rows_max, E, st, 1, 0, 0, 0, s,
                                   timer);
}

cudaError_t crt_row_exponents_batched(const double* X, int64_t ld, int tview, Dim rows, Dim K,
                                      const int64_t* rdev, int64_t rows_max, int32_t* E,
                                      DevState* st, int nz, int64_t zX, int64_t zR, int64_t zE,
                                      cudaStream_t s, KernelTimer* timer, const ZNest* znp) {
  if (nz < 1 || nz > 65535) return cudaErrorInvalidValue;
  // operands of separate problems have their own states; the nodes of one
  // matrix (zR = 0) share its state
  const int64_t zSt = (nz > 1 && zR != 0) ? 1 : 0;
  const ZNest zn = znp ? *znp : ZNest{1, 0, 0};
  if (zn.nzi < 1) return cudaErrorInvalidValue;
  return timer->run(KT_SPLIT, s, [&] {
    if (!tview)
      row_expo_kernel<<<dim3((unsigned)((rows_max * 32 + 255) / 256), 1, (unsigned)nz), 256, 0,
                        s>>>(X, ld, 0, rows, K, rdev, E, st, zX, zR, zE, zSt, zn);
    else
      row_expo_kernel<<<dim3((unsigned)((rows_max + 31) / 32), 16, (unsigned)nz), 256, 0, s>>>(
          X, ld, 1, rows, K, rdev, E, st, zX, zR, zE, zSt, zn);
    return cudaGetLastError();
  });
}

cudaError_t crt_split(const double* X, int64_t ld, int tview, Dim rows, Dim K, const int64_t* rdev,
                      int64_t rows_max, int64_t kpad, const int32_t* E, int n_mod, int beta,
                      void* out, cudaStream_t s, KernelTimer* timer, bool trim_k) {
  return crt_split_batched(X, ld, tview, rows, K, rdev, rows_max, kpad, E, n_mod, beta, out, 1, 0,
                           0, s, timer, nullptr, trim_k);
}

cudaError_t crt_split_batched(const double* X, int64_t ld, int tview, Dim rows, Dim K,
                              const int64_t* rdev, int64_t rows_max, int64_t kpad,
                              const int32_t* E, int n_mod, int beta, void* out, int nz,
                              int64_t zX, int64_t zR, cudaStream_t s, KernelTimer* timer,
                              const ZNest* znp, bool trim_k) {
  if (nz < 1 || nz > 65535 || rows_max % 32) return cudaErrorInvalidValue;
  const ZNest zn = znp ? *znp : ZNest{1, 0, 0};
  if (zn.nzi < 1) return cudaErrorInvalidValue;
  dim3 grid((unsigned)(kpad / 64), (unsigned)((rows_max + 31) / 32), (unsigned)nz);
  const int64_t zrow = nz > 1 ? rows_max : 0;
  return timer->run(KT_SPLIT, s, [&] {
    split_kernel<<<grid, 256, 0, s>>>(X, ld, tview, rows, K, rows_max, kpad, rdev, E, n_mod, beta,
                                      (bf16*)out, zX, zR, zrow, rows_max * nz, zn,
                                      trim_k ? 1 : 0);
    return cudaGetLastError();
  });
}

cudaError_t crt_mma(const void* SA, int64_t a_rows, int a_row0, const void* SB, int64_t b_rows,
                    int b_row0, int64_t kpad, int64_t kuse, int n_mod, Dim M, Dim N,
                    const int64_t* rdev, int lower, uint8_t* R, int64_t Mpad, int64_t Npad,
                    int32_t* status, cudaStream_t s, KernelTimer* timer, const GemmParams* fl,
                    int max_ctas, int blk, int bn, const BlockPlace* bplace,
                    const Dim* kdim) {
  const int64_t Mmax = M.max, Nmax = N.max;
  if (Mmax <= 0 || Nmax <= 0) return cudaSuccess;
  int BN = (Nmax >= 2048) ? 256 : (Nmax <= 32 ? 32 : 128);
  if (blk) {
    BN = (bn == 256 && blk % 256 == 0) ? 256 : 128;  // a tile never leaves its block
    // blocks that keep at most 32 columns (bplace) take 32-wide tiles
    if (bplace && bplace->N.max <= 32) BN = 32;
  }
  else if (bn == 128 || bn == 256) BN = bn;
  CUtensorMap ta, tb;
  if (!make_map(&ta, (const bf16*)SA, kpad, a_rows, n_mod, BM)) return cudaErrorInvalidValue;
  if (!make_map(&tb, (const bf16*)SB, kpad, b_rows, n_mod, BN)) return cudaErrorInvalidValue;
  MmaParams mp;
  std::memset(&mp, 0, sizeof(mp));
  mp.M = M;
  mp.N = N;
  mp.a_row0 = a_row0;
  mp.b_row0 = b_row0;
  mp.rdev = rdev;
  mp.nk = (int)((kuse + BK - 1) / BK);
  if (mp.nk < 1) mp.nk = 1;
  if (kdim && kdim->sel) {
    mp.kdev = 1;
    mp.Kd = *kdim;
  }
  mp.n_mod = n_mod;
  mp.lower = lower;
  mp.blk = blk;
  if (blk && bplace) {
    if (bplace->nzi < 1) return cudaErrorInvalidValue;
    mp.bdims = 1;
    mp.bnzi = bplace->nzi;
    mp.bzR = bplace->zR;
    mp.bzoff = bplace->zoff;
    mp.bM = bplace->M;
    mp.bN = bplace->N;
  }
  mp.R = R;
  mp.Mpad = Mpad;
  mp.Npad = Npad;
  mp.status = status;
  const int64_t wave = max_ctas > 0 ? max_ctas : 152;
  KernelTimer mt = *timer;
  mt.gemm = fl;
  mt.flops_mult = (double)n_mod;
  return mt.run(KT_MMA, s, [&] {
    if (BN == 256) return launch_mma<256, 4, false>(ta, tb, mp, Mmax, Nmax, wave, s);
    // a capped grid shares the SMs with concurrent work: fewer stages, less
    // shared memory per CTA
    if (BN == 32 && max_ctas > 0) return launch_mma<32, 4, false>(ta, tb, mp, Mmax, Nmax, wave, s);
    if (BN == 32) return launch_mma<32, 8, false>(ta, tb, mp, Mmax, Nmax, wave, s);
    return launch_mma<128, 6, false>(ta, tb, mp, Mmax, Nmax, wave, s);
  });
}

// The CRT tables of every moduli count, uploaded once per device (outside
// any stream capture: the first call of an argument set always runs
// directly); returns their device address, indexed by the moduli count.
// The address is kept for the life of the process, like the library's
// streams, events and graphs: it belongs to the device's primary context,
// so a reset of that context (cudaDeviceReset) between calls is not
// supported.
const crt::Consts* crt_consts_device() {
  static std::mutex mu;
  static std::vector<std::pair<int, const crt::Consts*>> done;
  std::lock_guard<std::mutex> lock(mu);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  for (auto& d : done)
    if (d.first == dev) return d.second;
  static crt::Consts host[crt::kMaxMod + 1];
  for (int k = 1; k <= crt::kMaxMod; ++k) crt::make_consts(k, &host[k]);
  if (cudaMemcpyToSymbol(g_crt_consts, host, sizeof(host)) != cudaSuccess) return nullptr;
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_crt_consts) != cudaSuccess || !ptr) return nullptr;
  done.push_back({dev, (const crt::Consts*)ptr});
  return (const crt::Consts*)ptr;
}

cudaError_t crt_reconstruct(const uint8_t* R, int64_t Mpad, int64_t Npad, Dim M, Dim N,
                            const int64_t* rdev, const int32_t* EA, const int32_t* EB, int betaA,
                            int betaB, double alpha, double beta, double* C, int64_t ldc,
                            int lower, int n_mod, cudaStream_t s, KernelTimer* timer, int blk,
                            const BlockPlace* bplace) {
  if (!crt_consts_device()) return cudaErrorInitializationError;
  if (blk && (n_mod > kRecWordsMaxMod || Npad != blk)) return cudaErrorInvalidValue;
  ReconParams rp;
  rp.R = R;
  rp.Mpad = Mpad;
  rp.Npad = Npad;
  rp.M = M;
  rp.N = N;
  rp.rdev = rdev;
  rp.EA = EA;
  rp.EB = EB;
  rp.betaA = betaA;
  rp.betaB = betaB;
  rp.alpha = alpha;
  rp.beta = beta;
  rp.C = C;
  rp.ldc = ldc;
  rp.lower = lower;
  rp.blk = blk;
  rp.bdims = 0;
  rp.bnzi = 1;
  rp.zC = (int64_t)blk * ldc;
  rp.zCo = 0;
  rp.zoff = 0;
  rp.bzR = 0;
  rp.bM = rp.bN = hdim(0);
  if (blk && bplace) {
    if (bplace->nzi < 1) return cudaErrorInvalidValue;
    rp.bdims = 1;
    rp.bnzi = bplace->nzi;
    rp.bzR = bplace->zR;
    rp.zCo = bplace->zCo;
    rp.zC = bplace->zC;
    rp.zoff = bplace->zoff;
    rp.bM = bplace->M;
    rp.bN = bplace->N;
  }
  // small outputs (factorisation panels): latency-bound, four lanes per output
  // (block-diagonal outputs always take the word-wise kernel)
  const bool small = !blk && M.max * N.max <= ((int64_t)1 << 16);
  // outputs of at most 32 columns (the batched factorisation's panels): eight
  // threads per row, so that no lane idles
  const bool narrow = N.max <= 32;
  const dim3 gw((unsigned)((N.max + kRecWCols - 1) / kRecWCols),
                (unsigned)((M.max + kRecWRows - 1) / kRecWRows));
  const dim3 gn(1, (unsigned)((M.max + 31) / 32));
  return timer->run(KT_RECON, s, [&] {
    if (small)
      reconstruct_split_kernel<<<grid1d(M.max * N.max * kRecLanes, 256), 256, 0, s>>>(rp, n_mod);
    else if (n_mod <= kRecWords4MaxMod && narrow)
      reconstruct_words_kernel<4, 8><<<gn, 256, 0, s>>>(rp, n_mod);
    else if (n_mod <= kRecWords4MaxMod)
      reconstruct_words_kernel<4, 32><<<gw, 256, 0, s>>>(rp, n_mod);
    else if (n_mod <= kRecWordsMaxMod && narrow)
      reconstruct_words_kernel<5, 8><<<gn, 256, 0, s>>>(rp, n_mod);
    else if (n_mod <= kRecWordsMaxMod)
      reconstruct_words_kernel<5, 32><<<gw, 256, 0, s>>>(rp, n_mod);
    else
      reconstruct_kernel<<<grid1d(M.max * ((N.max + kRecW - 1) / kRecW), 256), 256, 0, s>>>(
          rp, n_mod);
    return cudaGetLastError();
  });
}

size_t split_workspace_bytes(int64_t Mmax, int64_t Nmax, int64_t Kmax, bool same_operand) {
  const int64_t kpad = round_up(Kmax > 0 ? Kmax : 1, BK);
  const int64_t mpad = round_up(Mmax > 0 ? Mmax : 1, BM);
  const int64_t npad = round_up(Nmax > 0 ? Nmax : 1, 256);
  size_t b = 0;
  auto add = [&](size_t x) { b = (b + 1023) / 1024 * 1024 + x; };
  add(sizeof(bf16) * 2 * (size_t)mpad * (size_t)kpad);
  if (!same_operand) add(sizeof(bf16) * 2 * (size_t)npad * (size_t)kpad);
  add(sizeof(int32_t) * (size_t)(mpad + npad));
  return b + 1024;
}

// Split-precision product (BF16x3, FP32 accumulation): reduced accuracy,
// about 2^-16 relative per term.
cudaError_t launch_split_gemm(const CrtGemm& g, cudaStream_t s, KernelTimer* timer) {
  const GemmParams& p = g.p;
  const int64_t Mmax = p.M.max, Nmax = p.N.max, Kmax = p.K.max;
  if (Mmax <= 0 || Nmax <= 0) return cudaSuccess;
  const int64_t kpad = round_up(Kmax > 0 ? Kmax : 1, BK);
  const int64_t mpad = round_up(Mmax, BM);
  const int64_t npad = round_up(Nmax, 256);
  const bool same = g.same_operand;
  char* w = (char*)g.ws;
  size_t off = 0;
  auto take = [&](size_t x) {
    off = (off + 1023) / 1024 * 1024;
    char* q = w + off;
    off += x;
    return q;
  };
  bf16* SA = (bf16*)take(sizeof(bf16) * 2 * (size_t)mpad * (size_t)kpad);
  bf16* SB = same ? SA : (bf16*)take(sizeof(bf16) * 2 * (size_t)npad * (size_t)kpad);
  int32_t* EA = (int32_t*)take(sizeof(int32_t) * (size_t)(mpad + npad));
  int32_t* EB = same ? EA : EA + mpad;
  if (off > g.ws_bytes) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(EA, 0, sizeof(int32_t) * (size_t)(mpad + npad), s);
  if (e != cudaSuccess) return e;
  auto split = [&](const double* X, int64_t ld, int tview, Dim rows, int64_t rows_max, int32_t* E,
                   bf16* S) -> cudaError_t {
    cudaError_t err = crt_row_exponents(X, ld, tview, rows, p.K, p.rdev, rows_max, E, g.st, s, timer);
    if (err != cudaSuccess) return err;
    dim3 grid((unsigned)(kpad / 32), (unsigned)((rows_max + 31) / 32));
    return timer->run(KT_SPLIT, s, [&] {
      split3_kernel<<<grid, 256, 0, s>>>(X, ld, tview, rows, p.K, rows_max, kpad, p.rdev, E, S);
      return cudaGetLastError();
    });
  };
  e = split(p.A, p.lda, g.transA ? 1 : 0, p.M, mpad, EA, SA);
  if (e == cudaSuccess && !same) e = split(p.B, p.ldb, g.transB ? 0 : 1, p.N, npad, EB, SB);
  if (e != cudaSuccess) return e;
  CUtensorMap ta, tb;
  if (!make_map(&ta, SA, kpad, mpad, 2, BM)) return cudaErrorInvalidValue;
  if (!make_map(&tb, SB, kpad, same ? mpad : npad, 2, 128)) return cudaErrorInvalidValue;
  MmaParams mp;
  std::memset(&mp, 0, sizeof(mp));
  mp.M = p.M;
  mp.N = p.N;
  mp.rdev = p.rdev;
  mp.nk = (int)(kpad / BK);
  mp.n_mod = 1;

  mp.lower = p.lower;
  mp.status = &g.st->status;
  mp.C = p.C;
  mp.ldc = p.ldc;
  mp.EA = EA;
  mp.EB = EB;
  mp.alpha = p.alpha;
  mp.beta = p.beta;
  KernelTimer mt = *timer;
  mt.gemm = &g.p;
  mt.flops_mult = 3.0;
  return mt.run(KT_MMA, s,
                [&] { return launch_mma<128, 3, true>(ta, tb, mp, Mmax, Nmax, 152, s); });
}

cudaError_t launch_crt_gemm(const CrtGemm& g, cudaStream_t s, KernelTimer* timer) {
  const GemmParams& p = g.p;
  const int64_t Mmax = p.M.max, Nmax = p.N.max, Kmax = p.K.max;
  if (Mmax <= 0 || Nmax <= 0) return cudaSuccess;
  if (Kmax > 4096) return cudaErrorInvalidValue;  // exactness bound of the FP32 sums
  const int n_mod = crt_moduli_for(Kmax, g.betaA, g.betaB);
  if (n_mod < 0) return cudaErrorInvalidValue;
  const int64_t kpad = round_up(Kmax > 0 ? Kmax : 1, BK);
  const int64_t mpad = round_up(Mmax, BM);
  const int64_t npad = round_up(Nmax, 256);
  const bool same = g.same_operand;
  char* w = (char*)g.ws;
  size_t off = 0;
  auto take = [&](size_t x) {
    off = (off + 1023) / 1024 * 1024;
    char* q = w + off;
    off += x;
    return q;
  };
  bf16* SA = (bf16*)take(sizeof(bf16) * (size_t)n_mod * (size_t)mpad * (size_t)kpad);
  bf16* SB = same ? SA : (bf16*)take(sizeof(bf16) * (size_t)n_mod * (size_t)npad * (size_t)kpad);
  uint8_t* R = (uint8_t*)take((size_t)n_mod * (size_t)mpad * (size_t)npad);
  int32_t* EA = (int32_t*)take(sizeof(int32_t) * (size_t)(mpad + npad));
  int32_t* EB = same ? EA : EA + mpad;
  if (off > g.ws_bytes) return cudaErrorInvalidValue;

  cudaError_t e = cudaMemsetAsync(EA, 0, sizeof(int32_t) * (size_t)(mpad + npad), s);
  if (e != cudaSuccess) return e;
  // op(A): rows x K; transA: element (i,k) at A[k*lda + i].  op(B) is K x N;
  // its N x K view: element (j,k) = transB ? B[j*ldb + k] : B[k*ldb + j].
  // a device-side K: the residue planes end at its last block and the
  // product sums only up to there
  const bool kdev = p.K.sel != 0;
  e = crt_row_exponents(p.A, p.lda, g.transA ? 1 : 0, p.M, p.K, p.rdev, mpad, EA, g.st, s, timer);
  if (e == cudaSuccess)
    e = crt_split(p.A, p.lda, g.transA ? 1 : 0, p.M, p.K, p.rdev, mpad, kpad, EA, n_mod, g.betaA,
                  SA, s, timer, kdev);
  if (e == cudaSuccess && !same) {
    e = crt_row_exponents(p.B, p.ldb, g.transB ? 0 : 1, p.N, p.K, p.rdev, npad, EB, g.st, s, timer);
    if (e == cudaSuccess)
      e = crt_split(p.B, p.ldb, g.transB ? 0 : 1, p.N, p.K, p.rdev, npad, kpad, EB, n_mod, g.betaB,
                    SB, s, timer, kdev);
  }
  if (e != cudaSuccess) return e;
  e = crt_mma(SA, mpad, 0, SB, same ? mpad : npad, 0, kpad, Kmax, n_mod, p.M, p.N, p.rdev, p.lower,
              R, mpad, npad, &g.st->status, s, timer, &g.p, 0, 0, 0, nullptr,
              kdev ? &p.K : nullptr);
  if (e != cudaSuccess) return e;
  return crt_reconstruct(R, mpad, npad, p.M, p.N, p.rdev, EA, EB, g.betaA,
                         same ? g.betaA : g.betaB, p.alpha, p.beta, p.C, p.ldc, p.lower, n_mod, s,
                         timer);
}

}  // namespace cpinv
