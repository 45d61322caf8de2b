// Host-side launchers of the cpinv kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cpinv {

// ---------------------------------------------------------------------------
// Kernel classes for tracing, and the hook every launcher goes through
// (implemented in capi.cu).
// ---------------------------------------------------------------------------
enum : int {
  KT_GEMM_FP64 = 0,  // dgemm_kernel
  KT_MMA = 1,        // crt_mma_kernel (tcgen05)
  KT_DIAG = 2,       // diag_factor_kernel
  KT_AUX = 3,        // small O(n^2) kernels
  KT_SPLIT = 4,      // residue split of the operands
  KT_RECON = 5,      // CRT reconstruction
  KT_PANEL = 6,      // chol_panel_exact_kernel (fused panel of the exact factorisation)
  KT_COUNT = 7
};

void trace_count();
bool trace_on();
int trace_begin(cudaStream_t s);
void trace_end(int rec, cudaStream_t s, int kind, const GemmParams* g, double flops_mult);

struct KernelTimer {
  const GemmParams* gemm = nullptr;  // flops of the MMA launches come from its dims
  double flops_mult = 1.0;           // e.g. the number of moduli
  template <class F>
  cudaError_t run(int kind, cudaStream_t s, F&& f) {
    trace_count();
    if (!trace_on()) return f();
    const int rec = trace_begin(s);
    cudaError_t e = f();
    trace_end(rec, s, kind,
              kind == KT_MMA || kind == KT_GEMM_FP64 || kind == KT_DIAG || kind == KT_PANEL ? gemm
                                                                                          : nullptr,
              flops_mult);
    return e;
  }
};

// While alive, calls on this thread run their kernels directly (no CUDA-graph
// capture or replay: instantiating a graph may allocate).
struct NoGraphScope {
  NoGraphScope();
  ~NoGraphScope();
};
bool graph_replay_allowed();  // CUDA graphs on, no NoGraphScope, no tracing
void launches_add(int64_t n);  // kernels launched through a graph replay
// flop counts of traced launches whose dims read the DevState at rdev
cudaError_t trace_finish(cudaStream_t s, const int64_t* rdev);

// One FP64-accurate product in the residue (exact-slice) arithmetic.
struct CrtGemm {
  GemmParams p;       // C = alpha op(A) op(B) + beta C  (dims may depend on the device rank)
  bool transA, transB;
  bool same_operand;  // op(B) is op(A)' (symmetric products): split once
  int betaA, betaB;   // integer bits of the scaled operands (<= 62)
  void* ws;           // scratch, crt_workspace_bytes() bytes, 1024-aligned
  size_t ws_bytes;
  DevState* st;
};
size_t crt_workspace_bytes(int64_t Mmax, int64_t Nmax, int64_t Kmax, int n_mod, bool same_operand);
cudaError_t launch_crt_gemm(const CrtGemm& g, cudaStream_t s, KernelTimer* timer);
int crt_moduli_for(int64_t Kmax, int betaA, int betaB);
size_t split_workspace_bytes(int64_t Mmax, int64_t Nmax, int64_t Kmax, bool same_operand);
cudaError_t launch_split_gemm(const CrtGemm& g, cudaStream_t s, KernelTimer* timer);
int crt_block_k();  // K granularity of the residue planes (64)
namespace crt { struct Consts; }
const crt::Consts* crt_consts_device();  // CRT tables [moduli count], device address
int crt_block_m();  // rows of an output tile (128)
// The three stages of an exact product, for callers that keep residues:
//   row exponents (atomicMax into a zeroed array), residue planes
//   S[j][row][k] (BF16, rows_max x kpad per modulus), the tensor-core
//   products mod p_j into R[j][row][col], and the CRT reconstruction.
cudaError_t crt_row_exponents(const double* X, int64_t ld, int tview, Dim rows, Dim K,
                              const int64_t* rdev, int64_t rows_max, int32_t* E, DevState* st,
                              cudaStream_t s, KernelTimer* timer);
// trim_k: the planes are written only up to the last BK block inside K (a
// product that reads them must then sum only those blocks: crt_mma's kdim).
cudaError_t crt_split(const double* X, int64_t ld, int tview, Dim rows, Dim K, const int64_t* rdev,
                      int64_t rows_max, int64_t kpad, const int32_t* E, int n_mod, int beta,
                      void* out, cudaStream_t s, KernelTimer* timer, bool trim_k = false);
// Largest moduli count of a block-diagonal reconstruction (crt_reconstruct
// with blk > 0).
constexpr int kRecBlockMaxMod = 22;
// Placement of the blocks of a block-diagonal output, block z = zo nzi + zi
// (zo: the problem, zi: a block inside it): block z keeps its rows i < M and
// columns j < N (each with zi zoff added to its offset, the rank read at
// rdev + zo zR) and writes them to C + zo zCo + zi zC + i ldc + j.
struct BlockPlace {
  Dim M, N;
  int64_t zoff, zC;
  int32_t nzi = 1;
  int64_t zR = 0, zCo = 0;
};
// blk > 0: block-diagonal product (the Gram matrices of a batch stacked
// along M = N): only the tiles inside the blk x blk diagonal blocks, R holds
// [n_mod][Mpad][blk]; bn: output tile width (0 = by size; 128 or 256);
// bplace: the tiles past a block's rows or columns (bplace->M, N) skipped;
// kdim: a device-side K (at most kuse): the BK blocks past it are not summed.
cudaError_t crt_mma(const void* SA, int64_t a_rows, int a_row0, const void* SB, int64_t b_rows,
                    int b_row0, int64_t kpad, int64_t kuse, int n_mod, Dim M, Dim N,
                    const int64_t* rdev, int lower, uint8_t* R, int64_t Mpad, int64_t Npad,
                    int32_t* status, cudaStream_t s, KernelTimer* timer, const GemmParams* fl,
                    int max_ctas = 0, int blk = 0, int bn = 0,
                    const BlockPlace* bplace = nullptr, const Dim* kdim = nullptr);
// blk > 0: the block-diagonal output of crt_mma (rows Mpad, Npad = blk),
// written to C (row i, its block's column j) with EB per block; bplace: the
// blocks placed and clipped as it says (default: block z at rows z blk of C,
// every row and column kept).
cudaError_t crt_reconstruct(const uint8_t* R, int64_t Mpad, int64_t Npad, Dim M, Dim N,
                            const int64_t* rdev, const int32_t* EA, const int32_t* EB, int betaA,
                            int betaB, double alpha, double beta, double* C, int64_t ldc,
                            int lower, int n_mod, cudaStream_t s, KernelTimer* timer,
                            int blk = 0, const BlockPlace* bplace = nullptr);
// Batches of nz operands (z-major), z = zo nzi + zi (zn; default nzi = 1):
// operand z at X + zo zX + zi zXi with its dims read at rdev + zo zR and
// zi zoff added to their offsets; its exponents and residue rows follow one
// another (rows z rows_max .. in E and in the planes, plane rows =
// nz rows_max).  zR = 0: the operands are blocks of one matrix and share its
// state.
cudaError_t crt_row_exponents_batched(const double* X, int64_t ld, int tview, Dim rows, Dim K,
                                      const int64_t* rdev, int64_t rows_max, int32_t* E,
                                      DevState* st, int nz, int64_t zX, int64_t zR, int64_t zE,
                                      cudaStream_t s, KernelTimer* timer,
                                      const ZNest* zn = nullptr);
cudaError_t crt_split_batched(const double* X, int64_t ld, int tview, Dim rows, Dim K,
                              const int64_t* rdev, int64_t rows_max, int64_t kpad,
                              const int32_t* E, int n_mod, int beta, void* out, int nz,
                              int64_t zX, int64_t zR, cudaStream_t s, KernelTimer* timer,
                              const ZNest* zn = nullptr, bool trim_k = false);

// chol_queue.cu: the factorisations of a batch in one persistent launch
// fed by a device task queue (tasks on 32 x 32 tiles, listed in dependency
// order by the host; see the file's comment).
enum : int32_t { kQDiag = 0, kQSolve = 1, kQUpd = 2 };
struct QueueTask {
  int32_t kind;  // kQDiag, kQSolve, kQUpd
  int32_t z;     // problem (within the bucket)
  int16_t p;     // panel
  int16_t i, j;  // block row / block column (SOLVE: i; UPD: i >= j)
  int16_t pad;
};
static_assert(sizeof(QueueTask) == 16, "QueueTask layout");
struct QueueFactor {
  double* A;          // problem z at A + z zA, row-major, ld np
  int64_t np, zA;
  int32_t sel;        // SEL_N: order n_z, Appendix tolerance; SEL_RANK: order r_z, tol 0
  int32_t spd;
  DevState* st;       // per problem
  uint8_t* acc;       // kept mask (spd = 0), acc + z zAcc
  int64_t zAcc;
  double* dinv;       // 1 / L_cc per column, dinv + z zDinv (np per problem)
  int64_t zDinv;
  int32_t* flags;     // per problem (zeroed): ver[nb][nb], solved[nb], diag[nb]
  int64_t zFlags;
  int32_t nb_max;     // blocks of np
  int32_t ntasks;
  const QueueTask* tasks;
  int32_t* head;      // [0] next task (zeroed), [1] abort flag (zeroed)
};
cudaError_t launch_chol_queue(const QueueFactor& q, int ctas, cudaStream_t s);
int chol_queue_ctas();  // CTAs of one wave on this device (0 on error)

// chol_exact.cu
cudaError_t launch_rowscale(const double* A, int64_t lda, Dim nd, const int64_t* rdev,
                            int64_t rows_max, int32_t* E, cudaStream_t s);
// One fused launch per panel of the exact-slice factorisation (update
// reconstruction, diagonal block, rows below, residue split).
struct PanelExactParams {
  const uint8_t* R;   // residues of the update of panel kn over columns 0 .. kb, R[j][row][col] (rows from kn)
  int64_t Mpad, Npad;
  int32_t has_update, n_upd;  // has_update = 0: the first launch (block 0 only); moduli count of the update
  int32_t has_bulk;   // kb > 0: R holds the part over columns 0 .. kb
  int32_t k_last;     // columns kb .. kn (<= 96) summed exactly in the kernel
  int64_t kb;
  const crt::Consts* consts;  // crt_consts_device()
  double* A;
  int64_t lda;
  Dim nd;
  const int64_t* rdev;
  int64_t ks;         // panel whose rows below its block are solved here (block factored by the previous launch)
  int64_t kn;         // ks + b: the block factored here
  int32_t b, spd;
  DevState* st;
  uint8_t* accepted;
  const double* dinv_prev;  // 1/T_cc of block ks
  double* dinv_next;        // 1/T_cc of block kn (written here)
  const int32_t* E;   // row scales (biased exponent bounds)
  int32_t n_mod, beta;  // residues of the factor: moduli count and bits
  __nv_bfloat16* RL;
  int64_t rl_rows, rl_kpad;
  int32_t nbr;        // CTAs 1..nbr solve the rows of block kn (chol_panel_exact_nbr)
  int32_t helpers;    // the next CTAs update block kn (chol_panel_exact_helpers)
  int64_t rows_target;  // st->panel_flag once this launch's block-row CTAs are done
  int64_t diag_target;  // st->diag_count once its helpers are done
};
// One CTA waits, bounded, on st->spare[0] >= 1 (nothing sets it): records
// ST_TIMEOUT in st->status after about a second and returns.
cudaError_t launch_wait_selftest(DevState* st, cudaStream_t s);
cudaError_t launch_chol_panel_exact(const PanelExactParams& p, cudaStream_t s);
int64_t chol_panel_exact_ctas(int64_t nmax, int64_t kn, int b);  // grid size of that launch
int chol_panel_exact_nbr(int b);      // block-row CTAs of a launch factoring a block of order b
int chol_panel_exact_helpers(int b);  // helper CTAs of that launch

// gemm_fp64.cu
cudaError_t launch_dgemm(const GemmParams& p, bool transA, bool transB, cudaStream_t s);

// chol.cu
cudaError_t launch_tol(const double* A, int64_t lda, int64_t n, double rel_tol, DevState* st,
                       cudaStream_t s);
// Diagonal block of panel k0 (b <= 32): factor in place, 1/L_cc into dinv[c]
// (0 for a rejected pivot), kept mask into accepted (spd = 0).  spd = 1:
// tolerance 0, every pivot must be kept (else ST_NUMERICAL), kept count
// added to st->rank_n.
cudaError_t launch_diag_factor(double* A, int64_t lda, Dim nd, int64_t k0, int b, DevState* st,
                               const int64_t* rdev, uint8_t* accepted, double* dinv, int spd,
                               cudaStream_t s);
// The same for a batch of nz equal-shaped problems (b <= 32); problem z uses
// A + z*zA etc., st[z] and the dims' device values of st[z].
struct DiagBatch {
  double* A;
  int64_t lda, zA;
  Dim nd;          // order of each problem's matrix
  int64_t k0;
  int32_t b, spd;
  DevState* st;
  uint8_t* accepted;
  int64_t zAcc;
  double* dinv;
  int64_t zDinv;
};
cudaError_t launch_diag_batched(const DiagBatch& p, int nz, cudaStream_t s);
// Rows below the diagonal block of panel k0: L(i, P) T' = A(i, P) by forward
// substitution against the factored block (in place).
cudaError_t launch_panel_solve(double* A, int64_t lda, Dim nd, const int64_t* rdev, int64_t k0,
                               int b, const double* dinv, cudaStream_t s);
struct PanelBatch {
  double* A;
  int64_t lda, zA;
  Dim nd;
  int64_t k0;
  int32_t b, pad;
  const double* dinv;
  int64_t zDinv;
  const DevState* st;
};
cudaError_t launch_panel_solve_batched(const PanelBatch& p, int nz, cudaStream_t s);
// Inverses of the b x b diagonal blocks of a lower-triangular matrix of
// order r = *rdev (b <= 32), Tinv[q] row-major b x b; batched form: problem z
// uses T + z*zT, rdev[z*zR], Tinv + z*zTinv.
cudaError_t launch_tri_block_inverse(const double* T, int64_t ld, int64_t nmax,
                                     const int64_t* rdev, int b, double* Tinv, cudaStream_t s);
cudaError_t launch_tri_block_inverse_batched(const double* T, int64_t ld, int64_t zT,
                                             int64_t nmax, const int64_t* rdev, int64_t zR, int b,
                                             double* Tinv, int64_t zTinv, int nz, cudaStream_t s);
cudaError_t launch_scan(const uint8_t* accepted, int64_t n, int32_t* colidx, DevState* st,
                        cudaStream_t s);
cudaError_t launch_gather(const double* Lfull, int64_t lda, int64_t n, const int32_t* colidx,
                          double* L, int64_t ldl, cudaStream_t s);
cudaError_t launch_tri_inv_init(double* W, int64_t ldw, int64_t nmax, const int64_t* rdev,
                                const double* Tinv, int b, cudaStream_t s);
cudaError_t launch_mirror(double* C, int64_t ldc, Dim nd, const int64_t* rdev, cudaStream_t s);
cudaError_t launch_copy_mask(const uint8_t* src, uint8_t* dst, int64_t n, cudaStream_t s);


// adjoint.cu (reverse pass of W = G+ F)
cudaError_t launch_pivot_lists(const uint8_t* acc, int64_t n, int32_t* pref, int32_t* sidx,
                               int32_t* didx, cudaStream_t s);
cudaError_t launch_pattern_mask(double* Lb, int64_t ld, int64_t n, const int32_t* pref,
                                const int64_t* rdev, cudaStream_t s);
cudaError_t launch_gather_rows(const double* src, int64_t lds, const int32_t* idx, int64_t n,
                               int count_rejected, const int64_t* rdev, double* dst, int64_t ldd,
                               cudaStream_t s);
cudaError_t launch_phi(double* P, int64_t ld, int64_t nmax, const int64_t* rdev, cudaStream_t s);
cudaError_t launch_sym_scatter(const double* ASS, int64_t lss, const double* ADS, int64_t lds,
                               const int32_t* colidx, const int32_t* pref, int64_t n, double* As,
                               int64_t lda, cudaStream_t s);

}  // namespace cpinv
