// C ABI of cpinv (declared in include/cpinv.h) and the host-side pipeline.
//
// Pipeline of one call (Appendix `geninv`, Theorem 1), all on one stream:
//   Gram        A = G'G (or G G' when m < n), lower triangle        [matmul]
//   tol         rel_tol * min positive diagonal entry, NaN/Inf flag  [tol_kernel]
//   Cholesky    panels: diag block (pivot tests) / panel solve / trailing update
//   compaction  prefix sum of the kept-pivot mask, gather of the kept columns
//   N = L'L     lower triangle                                        [matmul]
//   N = U U'    Cholesky with every pivot required (SPD)
//   W = U^-1    block rows: W_p. = -U_pp^-1 (U_p,<p W_<p,<p)        [matmul]
//   M = W'W     = N^-1 = (L'L)^-1                                     [matmul]
//   pinv:  X = L M, K = X X', G+ = K G'   (G+ = G' K when m < n)
//   lstsq: W = L (M (M (L' (G'F))))       (G' (L (M (M (L'F))))) when m < n)
// The numerical rank r never leaves the device until the optional read-back
// at the end: every launch after the pivot tests is sized for the largest
// possible r and reads r from device memory.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/cpinv.h"
#include "common.cuh"
#include "kernels.h"

namespace cpinv {
namespace {

struct Arena {
  char* base;
  size_t off;
  void* take(size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

// (a batched problem's own m or n is not known here: its bound `max` stands in)
int64_t eval_host(const Dim& d, int64_t r) {
  int64_t v = d.off + (d.sel == SEL_RANK ? r : d.sel == -SEL_RANK ? -r : d.sel ? d.max : 0);
  v = v < 0 ? 0 : v;
  return v > d.max ? d.max : v;
}

double gemm_flops(const Dim& Md, const Dim& Nd, const Dim& Kd, int lower, int64_t r) {
  const double M = (double)eval_host(Md, r), N = (double)eval_host(Nd, r), K = (double)eval_host(Kd, r);
  double elems = M * N;
  if (lower) elems = (M <= N) ? M * (M + 1) / 2 : N * (N + 1) / 2 + (M - N) * N;
  return 2.0 * elems * K;
}

// ---------------------------------------------------------------------------
// Tracing: events around every launch (when enabled) and a launch counter.
// ---------------------------------------------------------------------------
const char* const kKindName[KT_COUNT] = {"gemm_fp64", "tc_mma",          "diag_factor", "aux",
                                         "split",     "crt_reconstruct", "chol_panel"};

struct TraceRec {
  cudaEvent_t e0, e1;
  int kind;
  bool resolved;
  double flops;
  double mult;
  Dim M, N, K;
  int lower;
};

struct Tracer {
  bool on = false;
  std::vector<TraceRec> recs;
};
Tracer g_tr;
std::atomic<int64_t> g_launches{0};

// Resolves the flop counts of the records that depend on the device rank
// (called at the end of each traced call, while the workspace is alive).
cudaError_t trace_resolve(cudaStream_t s, const int64_t* rdev) {
  if (!g_tr.on) return cudaSuccess;
  int64_t r = 0;
  cudaError_t e = cudaMemcpyAsync(&r, rdev, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  for (auto& t : g_tr.recs)
    if (!t.resolved) {
      t.flops = t.mult * gemm_flops(t.M, t.N, t.K, t.lower, r);
      t.resolved = true;
    }
  return cudaSuccess;
}

}  // namespace

void trace_count() { g_launches.fetch_add(1, std::memory_order_relaxed); }
bool trace_on() { return g_tr.on; }
int trace_begin(cudaStream_t s) {
  TraceRec r{};
  if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) return -1;
  cudaEventRecord(r.e0, s);
  g_tr.recs.push_back(r);
  return (int)g_tr.recs.size() - 1;
}
void trace_end(int rec, cudaStream_t s, int kind, const GemmParams* g, double mult) {
  if (rec < 0) return;
  TraceRec& r = g_tr.recs[(size_t)rec];
  cudaEventRecord(r.e1, s);
  r.kind = kind;
  r.mult = mult;
  if (g) {
    r.M = g->M;
    r.N = g->N;
    r.K = g->K;
    r.lower = g->lower;
    r.resolved = false;
  } else {
    r.resolved = true;
    r.flops = 0.0;
  }
}

namespace {

enum Job {
  JOB_RANK = 0,
  JOB_PINV = 1,
  JOB_LSTSQ = 2,
  JOB_BACKWARD = 3,
  JOB_GRAM_LSTSQ = 4,
  JOB_FORWARD_SAVE = 5,     // W = G+ F, factors kept in a backward-sized state
  JOB_BACKWARD_STATE = 6,   // the reverse pass from that state
};

struct Plan {
  int64_t m, n, nA, k;
  bool trans;
  int b;
  int mode;
  double rel_tol;
  DevState* st;
  uint8_t* acc;
  int32_t* colidx;
  double* dinv;  // 1/L_cc of the current diagonal block(s) (0: rejected); two slots of 32
  double* Tinv;
  double* bufA;  // A -> L_full -> N -> U -> K
  double* bufL;  // compact L (nA x nA, r columns used)
  double* bufW;  // W = U^-1 -> X
  double* bufM;  // M
  double* Tmp;   // b x nA
  double* c1;    // lstsq: nA x k (also G'F)
  double* c2;
  double* c3;
  // reverse pass (JOB_BACKWARD)
  int32_t* pref;  // kept pivots among 0..i
  int32_t* sidx;  // kept pivot indices, in order
  int32_t* didx;  // rejected pivot indices, in order
  double* e[5];   // nA x k: c3, cbar3, cbar2, cbar1, Bbar
  double* Lb;     // nA x nA: Lbar
  double* Mb;     // Mbar
  double* LS;     // kept rows of L, then their Lbar
  double* LbS;
  double* LD;     // rejected rows of L, then their Lbar
  double* LbD;
  double* X;      // L_S^-1
  double* S1;     // scratch
  double* S2;
  void* crt;     // exact-slice scratch (residues, exponents)
  size_t crt_bytes;
};

// Where a product sits in the pipeline decides its arithmetic:
//  exact-slice mode: the Gram matrix from 62-bit integers (an exactly summed,
//    once-rounded G'G), the other large products from 53-bit integers (FP64
//    accuracy);
//  split mode: the Gram matrix and the chain (L M, X X', K G', the
//    least-squares products) in BF16x3 split precision, the products feeding
//    (L'L)^-1 as in exact-slice mode;
//  the pivot tests, square roots and diagonal blocks are FP64 in every mode.
enum Site { S_FP64 = 0, S_GRAM = 1, S_PROD = 2, S_CHAIN = 3 };
enum ProdKind { PK_FP64 = 0, PK_EXACT = 1, PK_SPLIT = 2 };

constexpr int64_t kCrtMaxK = 4096;  // exactness bound of one residue product

// Small products stay on the FP64 pipe: below 2MNK = 2^27 the residue split,
// tensor-core pass and reconstruction do not repay themselves.  The Gram
// matrix always takes the tensor-core form (its rounding is what the method
// amplifies).
int prod_kind(const Plan& p, Site site, int64_t Mmax, int64_t Nmax, int64_t Kmax) {
  if (p.mode == CPINV_MODE_FP64 || site == S_FP64) return PK_FP64;
  if (Mmax <= 0 || Nmax <= 0 || Kmax <= 0) return PK_FP64;
  const bool big = 2.0 * (double)Mmax * (double)Nmax * (double)Kmax >= (double)(1 << 27) &&
                   Kmax >= 128;
  if (site != S_GRAM && !big) return PK_FP64;
  if (p.mode == CPINV_MODE_SPLIT_BF16X3 && (site == S_GRAM || site == S_CHAIN)) return PK_SPLIT;
  return PK_EXACT;
}

size_t crt_need(const Plan& p, Site site, int64_t M, int64_t N, int64_t K, bool same) {
  const int pk = prod_kind(p, site, M, N, K);
  if (pk == PK_SPLIT) return split_workspace_bytes(M, N, K, same);
  if (pk != PK_EXACT) return 0;
  const int beta = site == S_GRAM ? 62 : 53;
  const int64_t Kc = K < kCrtMaxK ? K : kCrtMaxK;
  const int nm = crt_moduli_for(Kc, beta, beta);
  if (nm < 0) return 0;
  return crt_workspace_bytes(M, N, Kc, nm, same);
}

// Exact left-looking Cholesky (panel width <= 32, order <= 4096): residue
// planes of the factor RL[j][row][col], the update residues and row scales.
constexpr int kCholBits = 60;

struct CholLayout {
  int n_mod;
  int64_t rows, kpad;  // RL planes: rows x kpad per modulus
  size_t rl_bytes, r_bytes, e_bytes;
};

bool chol_exact_ok(const Plan& p) {
  return (p.mode == CPINV_MODE_EXACT_SLICE || p.mode == CPINV_MODE_SPLIT_BF16X3) && p.b <= 32 &&
         p.nA <= 4096 && p.nA > p.b;
}

CholLayout chol_layout(const Plan& p) {
  CholLayout L{};
  const int64_t bm = crt_block_m(), bk = crt_block_k();
  L.n_mod = crt_moduli_for(p.nA, kCholBits, kCholBits);
  L.rows = (p.nA + bm - 1) / bm * bm;
  L.kpad = (p.nA + bk - 1) / bk * bk;
  L.rl_bytes = 2 * (size_t)L.n_mod * (size_t)L.rows * (size_t)L.kpad;
  L.r_bytes = (size_t)L.n_mod * (size_t)L.rows * 256;
  L.e_bytes = sizeof(int32_t) * (size_t)L.rows;
  return L;
}

size_t chol_need(const Plan& p) {
  if (!chol_exact_ok(p)) return 0;
  const CholLayout L = chol_layout(p);
  return L.rl_bytes + 2 * L.r_bytes + L.e_bytes + 4 * 1024;
}

size_t crt_plan_bytes(const Plan& p, Job job) {
  const int64_t nA = p.nA, m = p.m, n = p.n;
  size_t need = crt_need(p, S_GRAM, nA, nA, p.trans ? n : m, true);
  need = chol_need(p) > need ? chol_need(p) : need;
  if (job == JOB_RANK) return need;
  auto mx = [&](size_t v) { need = v > need ? v : need; };
  mx(crt_need(p, S_PROD, nA, nA, nA, true));    // L'L, W'W
  mx(crt_need(p, S_PROD, nA, nA, nA, false));   // inverse blocks
  mx(crt_need(p, S_CHAIN, nA, nA, nA, true));   // X X'
  mx(crt_need(p, S_CHAIN, nA, nA, nA, false));  // L M
  if (job == JOB_PINV) mx(crt_need(p, S_CHAIN, n, m, nA, false));  // G+ = K G' or G' K
  if (job == JOB_LSTSQ || job == JOB_BACKWARD) {
    mx(crt_need(p, S_CHAIN, n, p.k, m, false));   // G'F (or G't)
    mx(crt_need(p, S_CHAIN, nA, p.k, nA, false)); // L'c, M c, L c
  }
  if (job == JOB_BACKWARD) {
    mx(crt_need(p, S_PROD, nA, nA, p.k, false));  // Wbar c3', B cbar1'
    mx(crt_need(p, S_PROD, nA, nA, nA, false));   // the r x r products
    mx(crt_need(p, S_CHAIN, m, n, n, false));     // Gbar = G (Abar + Abar')
    mx(crt_need(p, S_CHAIN, m, n, p.k, false));   // + F Bbar'
    mx(crt_need(p, S_CHAIN, m, p.k, n, false));   // Fbar = G Bbar
  }
  return need;
}

void carve(Plan& p, Arena& a, Job job) {
  const int64_t nA = p.nA, b = p.b;
  const int64_t nb = (nA + b - 1) / b;
  p.st = (DevState*)a.take(sizeof(DevState));
  p.crt_bytes = crt_plan_bytes(p, job);
  p.crt = p.crt_bytes ? a.take(p.crt_bytes) : nullptr;
  p.acc = (uint8_t*)a.take((size_t)(nA > 0 ? nA : 1));
  p.colidx = (int32_t*)a.take(sizeof(int32_t) * (size_t)(nA > 0 ? nA : 1));
  p.dinv = (double*)a.take(sizeof(double) * 64);  // two slots of 32
  p.bufA = (double*)a.take(sizeof(double) * (size_t)(nA * nA));
  if (job == JOB_RANK) return;
  p.Tinv = (double*)a.take(sizeof(double) * (size_t)(nb * b * b));
  p.bufL = (double*)a.take(sizeof(double) * (size_t)(nA * nA));
  p.bufW = (double*)a.take(sizeof(double) * (size_t)(nA * nA));
  p.bufM = (double*)a.take(sizeof(double) * (size_t)(nA * nA));
  p.Tmp = (double*)a.take(sizeof(double) * (size_t)(b * nA));
  if (job == JOB_LSTSQ || job == JOB_BACKWARD) {
    const int64_t rows = p.n > p.m ? p.n : p.m;
    p.c1 = (double*)a.take(sizeof(double) * (size_t)(rows * p.k));
    p.c2 = (double*)a.take(sizeof(double) * (size_t)(nA * p.k));
    p.c3 = (double*)a.take(sizeof(double) * (size_t)(nA * p.k));
  }
  if (job == JOB_BACKWARD) {
    p.pref = (int32_t*)a.take(sizeof(int32_t) * (size_t)nA);
    p.sidx = (int32_t*)a.take(sizeof(int32_t) * (size_t)nA);
    p.didx = (int32_t*)a.take(sizeof(int32_t) * (size_t)nA);
    for (auto& x : p.e) x = (double*)a.take(sizeof(double) * (size_t)(nA * p.k));
    double** sq[] = {&p.Lb, &p.Mb, &p.LS, &p.LbS, &p.LD, &p.LbD, &p.X, &p.S1, &p.S2};
    for (double** q : sq) *q = (double*)a.take(sizeof(double) * (size_t)(nA * nA));
  }
}

bool make_plan(Plan& p, int64_t m, int64_t n, int64_t k, const cpinv_opts* o) {
  cpinv_opts d;
  cpinv_default_opts(&d);
  if (!o) o = &d;
  p.m = m;
  p.n = n;
  p.k = k;
  p.trans = m < n;
  p.nA = p.trans ? m : n;
  p.b = o->panel ? o->panel : 32;
  p.mode = o->mode;
  p.rel_tol = o->rel_tol;
  if (p.b < 1 || p.b > 32 || 64 % p.b != 0) return false;  // a divisor of 64, at most 32
  if (!(p.rel_tol >= 0.0) || !std::isfinite(p.rel_tol)) return false;
  if (o->mode != CPINV_MODE_FP64 && o->mode != CPINV_MODE_EXACT_SLICE &&
      o->mode != CPINV_MODE_SPLIT_BF16X3)
    return false;
  return true;
}

size_t plan_bytes(Plan& p, Job job) {
  Arena a{nullptr, 0};
  carve(p, a, job);
  return a.off + 256;
}

struct Ctx {
  cudaStream_t s;
  const Plan* p;
  const int64_t* rdev() const { return &p->st->rank; }
};

#define CK(x)                                   \
  do {                                          \
    cudaError_t _e = (x);                       \
    if (_e != cudaSuccess) return CPINV_ERR_CUDA; \
  } while (0)

// Exact-slice product; K beyond the exactness bound of one residue product is
// cut into chunks whose results are added in FP64 (beta = 1 after the first).
cudaError_t crt_product(const GemmParams& g, bool ta, bool tb, int bits, bool same, void* ws,
                        size_t ws_bytes, DevState* st, cudaStream_t s) {
  const Dim K = g.K;
  for (int64_t k0 = 0; k0 < (K.max > 0 ? K.max : 1); k0 += kCrtMaxK) {
    CrtGemm cg;
    cg.p = g;
    const int64_t kmax = K.max - k0 < kCrtMaxK ? K.max - k0 : kCrtMaxK;
    cg.p.K = K.sel ? Dim{K.off - k0, kmax, K.sel, 0} : hdim(kmax < K.off - k0 ? kmax : K.off - k0);
    cg.p.A = ta ? g.A + k0 * g.lda : g.A + k0;
    cg.p.B = tb ? g.B + k0 : g.B + k0 * g.ldb;
    cg.p.beta = k0 == 0 ? g.beta : 1.0;
    cg.transA = ta;
    cg.transB = tb;
    cg.same_operand = same;
    cg.betaA = cg.betaB = bits;
    cg.ws = ws;
    cg.ws_bytes = ws_bytes;
    cg.st = st;
    KernelTimer t;
    cudaError_t e = launch_crt_gemm(cg, s, &t);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// C = alpha op(A) op(B) + beta C  in the plan's arithmetic (see Site).
cudaError_t matmul(const Ctx& c, Site site, const double* A, int64_t lda, bool ta, const double* B,
                   int64_t ldb, bool tb, double* C, int64_t ldc, Dim M, Dim N, Dim K,
                   double alpha, double beta, int lower) {
  GemmParams g;
  std::memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.C = C;
  g.lda = lda;
  g.ldb = ldb;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = alpha;
  g.beta = beta;
  g.rdev = c.rdev();
  g.lower = lower;
  g.pad = (C == A || C == B) ? 1 : 0;
  const Plan& p = *c.p;
  const int pk = prod_kind(p, site, M.max, N.max, K.max);
  if (pk == PK_FP64) {
    KernelTimer t;
    t.gemm = &g;
    return t.run(KT_GEMM_FP64, c.s, [&] { return launch_dgemm(g, ta, tb, c.s); });
  }
  const bool same = A == B && lda == ldb && ta != tb;
  if (pk == PK_SPLIT) {
    CrtGemm sg;
    sg.p = g;
    sg.transA = ta;
    sg.transB = tb;
    sg.same_operand = same;
    sg.betaA = sg.betaB = 0;
    sg.ws = p.crt;
    sg.ws_bytes = p.crt_bytes;
    sg.st = p.st;
    KernelTimer t;
    return launch_split_gemm(sg, c.s, &t);
  }
  return crt_product(g, ta, tb, site == S_GRAM ? 62 : 53, same, p.crt, p.crt_bytes, p.st, c.s);
}

// Tracing of a diagonal-block launch: its algorithmic work is the block
// factorisation and the block inverse, (2/3) bw^3 flops with bw = the block
// order (clamped to the device rank when factoring N).
struct DiagTimer {
  GemmParams g;
  KernelTimer t;
  template <class F>
  cudaError_t run(int kind, cudaStream_t s, F&& f) {
    t.gemm = &g;
    return t.run(kind, s, f);
  }
};
DiagTimer diag_timer(const Ctx& c, int64_t k0, int b, int spd) {
  DiagTimer d;
  std::memset(&d.g, 0, sizeof(d.g));
  const Dim bw = spd ? rdim(-k0, b) : hdim(c.p->nA - k0 < b ? c.p->nA - k0 : b);
  d.g.M = d.g.N = d.g.K = bw;
  d.g.lower = 1;
  d.g.rdev = c.rdev();
  d.t.flops_mult = 2.0 / 3.0;
  return d;
}

// Blocked full-rank Cholesky, in place on the lower triangle of a (ld = lda).
// spd = 0: order nA (host), pivot test against the Appendix tolerance, mask
//          written to acc.  spd = 1: order r (device), tolerance 0, and the
//          inverses of the b x b diagonal blocks stored in Tinv at the end.
int factor(const Ctx& c, double* a, int64_t lda, int spd) {
  const Plan& p = *c.p;
  const int64_t nA = p.nA;
  const int b = p.b;
  const Dim nd = spd ? rdim(0, nA) : hdim(nA);
  for (int64_t k0 = 0; k0 < nA; k0 += b) {
    CK(diag_timer(c, k0, b, spd).run(KT_DIAG, c.s, [&] {
      return launch_diag_factor(a, lda, nd, k0, b, p.st, c.rdev(), spd ? nullptr : p.acc, p.dinv,
                                spd, c.s);
    }));
    if (k0 + b >= nA) continue;
    // panel below the block: forward substitution against the block factor
    CK(KernelTimer().run(KT_AUX, c.s, [&] {
      return launch_panel_solve(a, lda, nd, c.rdev(), k0, b, p.dinv, c.s);
    }));
    double* panel = a + (k0 + b) * lda + k0;
    double* trail = a + (k0 + b) * lda + (k0 + b);
    Dim below, bw;
    if (spd) {
      below = rdim(-(k0 + b), nA - k0 - b);
      bw = rdim(-k0, b);
    } else {
      below = hdim(nA - k0 - b);
      bw = hdim(b);
    }
    // trailing update, lower triangle
    CK(matmul(c, S_FP64, panel, lda, false, panel, lda, true, trail, lda, below, below, bw, -1.0,
              1.0, 1));
  }
  if (spd)
    CK(KernelTimer().run(KT_AUX, c.s, [&] {
      return launch_tri_block_inverse(a, lda, nA, c.rdev(), b, p.Tinv, c.s);
    }));
  return CPINV_OK;
}

// CTAs of a fused panel launch that share the update of its diagonal block
constexpr int64_t kPanelHelpers = 9;

// A second library stream per device, with the events of the look-ahead
// (reused cyclically: each wait is enqueued right after the record it
// refers to, before that event is recorded again).
constexpr int kSideEvents = 4;
// CTAs of the look-ahead residue product: it overlaps the previous panel's
// launch, which needs free SMs for its row CTAs
constexpr int kLookaheadCtas = 152;
struct SideStream {
  int device;
  std::mutex mu;  // one enqueuing thread at a time (the events are shared)
  cudaStream_t s;
  cudaEvent_t fork, join, mma[kSideEvents], done[kSideEvents];
};
std::mutex g_side_mu;
std::vector<SideStream*> g_side;

SideStream* side_stream() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_side_mu);
  for (auto* x : g_side)
    if (x->device == dev) return x;
  auto* x = new SideStream();
  x->device = dev;
  // the highest priority: when a look-ahead product and a panel launch become
  // ready together, the product's CTAs are placed first (one per SM), and the
  // panel's CTAs fill the room left beside them
  int lo = 0, hi = 0;
  bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&x->s, cudaStreamNonBlocking, hi) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&x->fork, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&x->join, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < kSideEvents && ok; ++i) {
    ok = cudaEventCreateWithFlags(&x->mma[i], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&x->done[i], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    delete x;
    return nullptr;
  }
  g_side.push_back(x);
  return x;
}

// Exact-slice left-looking variant of factor() (see chol_exact.cu).
int factor_exact(const Ctx& c, double* a, int64_t lda, int spd) {
  const Plan& p = *c.p;
  const int64_t nA = p.nA;
  const int b = p.b;
  const CholLayout Ly = chol_layout(p);
  char* base = (char*)p.crt;
  size_t off = 0;
  auto take = [&](size_t x) {
    off = (off + 1023) / 1024 * 1024;
    char* q = base + off;
    off += x;
    return q;
  };
  void* RL = take(Ly.rl_bytes);
  uint8_t* Rbuf[2] = {(uint8_t*)take(Ly.r_bytes), (uint8_t*)take(Ly.r_bytes)};
  int32_t* E = (int32_t*)take(Ly.e_bytes);
  if (off > p.crt_bytes) return CPINV_ERR_WORKSPACE;
  const Dim nd = spd ? rdim(0, nA) : hdim(nA);
  KernelTimer t;
  CK(t.run(KT_AUX, c.s, [&] { return launch_rowscale(a, lda, nd, c.rdev(), Ly.rows, E, c.s); }));
  CK(cudaMemsetAsync(RL, 0, Ly.rl_bytes, c.s));
  const crt::Consts* consts = crt_consts_device();
  if (!consts) return CPINV_ERR_CUDA;
  SideStream* side = side_stream();
  if (!side) return CPINV_ERR_CUDA;
  std::lock_guard<std::mutex> side_lock(side->mu);
  cudaStream_t s2 = side->s;
  CK(cudaEventRecord(side->fork, c.s));
  CK(cudaStreamWaitEvent(s2, side->fork, 0));
  const int64_t kblk = crt_block_k();
  const int nbr = chol_panel_exact_nbr(b), helpers = chol_panel_exact_helpers(b);
  // this factorisation's completion counters start at zero
  CK(cudaMemsetAsync(&p.st->panel_flag, 0, 2 * sizeof(int64_t), c.s));
  int64_t rows_target = 0, diag_target = 0;
  PanelExactParams pp;
  std::memset(&pp, 0, sizeof(pp));
  pp.Mpad = Ly.rows;
  pp.Npad = 256;
  pp.n_upd = Ly.n_mod;
  pp.consts = consts;
  pp.A = a;
  pp.lda = lda;
  pp.nd = nd;
  pp.rdev = c.rdev();
  pp.b = b;
  pp.spd = spd;
  pp.st = p.st;
  pp.accepted = spd ? nullptr : p.acc;
  pp.E = E;
  pp.n_mod = Ly.n_mod;
  pp.beta = kCholBits;
  pp.RL = (__nv_bfloat16*)RL;
  pp.rl_rows = Ly.rows;
  pp.rl_kpad = Ly.kpad;
  pp.nbr = nbr;
  pp.helpers = helpers;
  // 1/T_cc of block j in slot j & 1 (the launch that solves against block j
  // runs while the next block is factored)
  auto dinv_slot = [&](int64_t j) { return p.dinv + 32 * (j & 1); };
  // Launch L(-1) factors block 0; launch L(q), q = 0 .. np - 2, solves the
  // rows below block q and factors block q + 1 (see chol_exact.cu).  The
  // update of panel q + 1 that L(q) applies splits into the columns 0 .. kb,
  // whose residue product runs on the second stream once L(q - 2) is done
  // (while L(q - 1) runs; kb, a multiple of the residue planes' K block, is
  // at most the first column of panel q - 1), and the last columns kb .. kn,
  // summed exactly inside L(q).  Two residue buffers alternate.
  const int64_t np = (nA + b - 1) / b;
  {
    pp.has_update = 0;
    pp.ks = -b;
    pp.kn = 0;
    pp.dinv_next = dinv_slot(0);
    DiagTimer pt = diag_timer(c, 0, b, spd);
    CK(pt.run(KT_PANEL, c.s, [&] { return launch_chol_panel_exact(pp, c.s); }));
    CK(cudaEventRecord(side->done[0], c.s));
  }
  for (int64_t q = 0; q + 1 < np; ++q) {
    const int64_t ks = q * b, kn = ks + b;
    const int64_t kb = q >= 1 ? (q - 1) * b / kblk * kblk : 0;
    uint8_t* R = Rbuf[q & 1];
    if (kb > 0) {
      // residues of L(kn:n, 0:kb) L(P, 0:kb)', exactly, from the residue planes,
      // once launch L(q - 2) (launch number q - 1) has finished
      CK(cudaStreamWaitEvent(s2, side->done[(q - 1) % kSideEvents], 0));
      const Dim M = spd ? rdim(-kn, nA - kn) : hdim(nA - kn);
      const Dim N = spd ? rdim(-kn, b) : hdim(nA - kn < b ? nA - kn : b);
      GemmParams fl;
      std::memset(&fl, 0, sizeof(fl));
      fl.M = M;
      fl.N = N;
      fl.K = spd ? rdim(0, kb) : hdim(kb);
      fl.rdev = c.rdev();
      CK(crt_mma(RL, Ly.rows, (int)kn, RL, Ly.rows, (int)kn, Ly.kpad, kb, Ly.n_mod, M, N,
                 c.rdev(), 0, R, Ly.rows, 256, &p.st->status, s2, &t, &fl, kLookaheadCtas));
      CK(cudaEventRecord(side->mma[q % kSideEvents], s2));
      CK(cudaStreamWaitEvent(c.s, side->mma[q % kSideEvents], 0));
    }
    pp.R = R;
    pp.has_update = 1;
    pp.has_bulk = kb > 0;
    pp.kb = kb;
    pp.k_last = (int32_t)(kn - kb);
    pp.ks = ks;
    pp.kn = kn;
    pp.dinv_prev = dinv_slot(q);
    pp.dinv_next = dinv_slot(q + 1);
    rows_target += nbr;
    diag_target += helpers;
    pp.rows_target = rows_target;
    pp.diag_target = diag_target;
    // traced work of the launch, in FP64-equivalent flops: for the rows
    // kn .. n, the forward substitution against block ks (b per entry) and
    // the exact sum over the last kn - kb columns (2 per term) --
    // 2 (n - kn) b (kn - kb + b / 2) -- which covers the block's own b^3/3
    // factorisation as well; the bulk columns 0 .. kb are the look-ahead
    // product's work
    DiagTimer pt;
    std::memset(&pt.g, 0, sizeof(pt.g));
    pt.g.M = spd ? rdim(-kn, nA - kn) : hdim(nA - kn);
    pt.g.N = hdim(b);
    pt.g.K = hdim(kn - kb + b / 2);
    pt.g.rdev = c.rdev();
    pt.t.flops_mult = 1.0;
    CK(pt.run(KT_PANEL, c.s, [&] { return launch_chol_panel_exact(pp, c.s); }));
    CK(cudaEventRecord(side->done[(q + 1) % kSideEvents], c.s));
  }
  // join the second stream back
  CK(cudaEventRecord(side->join, s2));
  CK(cudaStreamWaitEvent(c.s, side->join, 0));
  if (spd)
    CK(t.run(KT_AUX, c.s, [&] {
      return launch_tri_block_inverse(a, lda, nA, c.rdev(), b, p.Tinv, c.s);
    }));
  return CPINV_OK;
}

// Tolerance, full-rank Cholesky and compaction of the Gram matrix already in
// bufA (lower triangle).  Leaves L in bufL (compact) and r in st->rank.
int rank_from_gram(const Ctx& c, bool compact) {
  const Plan& p = *c.p;
  const int64_t nA = p.nA;
  CK(KernelTimer().run(KT_AUX, c.s,
                       [&] { return launch_tol(p.bufA, nA, nA, p.rel_tol, p.st, c.s); }));
  int rc = chol_exact_ok(p) ? factor_exact(c, p.bufA, nA, 0) : factor(c, p.bufA, nA, 0);
  if (rc) return rc;
  CK(KernelTimer().run(KT_AUX, c.s,
                       [&] { return launch_scan(p.acc, nA, p.colidx, p.st, c.s); }));
  if (compact)
    CK(KernelTimer().run(KT_AUX, c.s, [&] {
      return launch_gather(p.bufA, nA, nA, p.colidx, p.bufL, nA, c.s);
    }));
  return CPINV_OK;
}

// Gram, tolerance, full-rank Cholesky, compaction.  Leaves L in bufL (JOB_PINV
// / JOB_LSTSQ) and r in st->rank.
int front_rank(const Ctx& c, const double* G, int64_t ldg, bool compact) {
  const Plan& p = *c.p;
  const int64_t nA = p.nA;
  if (!p.trans)  // A = G'G
    CK(matmul(c, S_GRAM, G, ldg, true, G, ldg, false, p.bufA, nA, hdim(nA), hdim(nA), hdim(p.m),
              1.0, 0.0, 1));
  else  // A = G G'
    CK(matmul(c, S_GRAM, G, ldg, false, G, ldg, true, p.bufA, nA, hdim(nA), hdim(nA), hdim(p.n),
              1.0, 0.0, 1));
  return rank_from_gram(c, compact);
}

// Integer width of the triangular-inverse level products' operands: wider than
// the 53 bits of an FP64 significand, so that the small entries of a row of an
// ill-conditioned inverse keep as many bits as an FP64 product gives them.
constexpr int kLevelBits = 62;

// One product of a triangular-inverse level for all its nodes at once, in the
// exact-slice arithmetic (62-bit rows): node z (lo = 2 s z, mid = lo + s) forms
//   C_z = alpha A_z B_z,   A_z: rows mid.. x K, B_z: K x columns lo..,
// from the node-0 blocks A0, B0, C0 (ld nA; node z's blocks 2 s (nA + 1)
// further on), with the node-0 dims rows (of A and C), K and cols (of B and
// C) moving by -2s per node.  Both operands' residues are stacked node after
// node, so the level is one split per operand, one block-diagonal tensor-core
// product (blocks s x s, the nodes past the rank skipped) and one
// reconstruction writing each node's block in place.  False: the scratch is
// too small or the shape is outside the block product's limits (the caller
// then takes the per-node products).
bool level_product_fits(const Plan& p, int64_t s, int64_t nodes) {
  const int64_t bk = crt_block_k(), bm = crt_block_m();
  if (s % bm || s > kCrtMaxK || nodes < 1 || nodes > 65535) return false;
  const int nm = crt_moduli_for(s, kLevelBits, kLevelBits);
  if (nm < 1 || nm > kRecBlockMaxMod) return false;
  const int64_t kpad = (s + bk - 1) / bk * bk, tot = nodes * s;
  const size_t need = 2 * (2 * (size_t)nm * tot * kpad + 1024) + (size_t)nm * tot * s + 1024 +
                      2 * sizeof(int32_t) * (size_t)tot + 4096;
  return p.crt && need <= p.crt_bytes;
}

cudaError_t level_product(const Ctx& c, int64_t s, int64_t nodes, const double* A0, Dim rows,
                          Dim K, const double* B0, Dim cols, double* C0, double alpha) {
  const Plan& p = *c.p;
  const int64_t nA = p.nA, bk = crt_block_k();
  const int nm = crt_moduli_for(s, kLevelBits, kLevelBits);
  const int64_t kpad = (s + bk - 1) / bk * bk, tot = nodes * s;
  const int64_t zX = 2 * s * nA + 2 * s, zoff = -2 * s;
  char* w = (char*)p.crt;
  size_t off = 0;
  auto take = [&](size_t x) {
    off = (off + 1023) / 1024 * 1024;
    char* q = w + off;
    off += x;
    return q;
  };
  void* SA = take(2 * (size_t)nm * tot * kpad);
  void* SB = take(2 * (size_t)nm * tot * kpad);
  uint8_t* R = (uint8_t*)take((size_t)nm * tot * s);
  int32_t* EA = (int32_t*)take(sizeof(int32_t) * (size_t)tot);
  int32_t* EB = (int32_t*)take(sizeof(int32_t) * (size_t)tot);
  const int64_t* rdev = c.rdev();
  KernelTimer t;
  cudaError_t e = cudaMemsetAsync(EA, 0, (size_t)((char*)(EB + tot) - (char*)EA), c.s);
  if (e != cudaSuccess) return e;
  // A_z row-wise; B_z through its transpose (rows = the output's columns)
  const ZNest zn{(int32_t)nodes, zX, zoff};
  e = crt_row_exponents_batched(A0, nA, 0, rows, K, rdev, s, EA, p.st, (int)nodes, 0, 0, s, c.s,
                                &t, &zn);
  if (e == cudaSuccess)
    e = crt_row_exponents_batched(B0, nA, 1, cols, K, rdev, s, EB, p.st, (int)nodes, 0, 0, s,
                                  c.s, &t, &zn);
  if (e == cudaSuccess)
    e = crt_split_batched(A0, nA, 0, rows, K, rdev, s, kpad, EA, nm, kLevelBits, SA, (int)nodes,
                          0, 0, c.s, &t, &zn);
  if (e == cudaSuccess)
    e = crt_split_batched(B0, nA, 1, cols, K, rdev, s, kpad, EB, nm, kLevelBits, SB, (int)nodes,
                          0, 0, c.s, &t, &zn);
  if (e != cudaSuccess) return e;
  BlockPlace place;
  place.M = rows;
  place.N = cols;
  place.zoff = zoff;
  place.zC = zX;
  place.nzi = (int32_t)nodes;
  GemmParams fl;  // traced work: the nodes' s x s x s products
  std::memset(&fl, 0, sizeof(fl));
  fl.M = fl.N = hdim(s);
  fl.K = hdim(tot);
  e = crt_mma(SA, tot, 0, SB, tot, 0, kpad, s, nm, hdim(tot), hdim(tot), rdev, 0, R, tot, s,
              &p.st->status, c.s, &t, &fl, 0, (int)s, 0, &place);
  if (e != cudaSuccess) return e;
  return crt_reconstruct(R, tot, s, hdim(tot), hdim(s), rdev, EA, EB, kLevelBits, kLevelBits,
                         alpha, 0.0, C0, nA, 0, nm, c.s, &t, (int)s, &place);
}

// W = U^-1 for the lower-triangular U (order r <= nA, ld nA), given the
// inverted b x b diagonal blocks already in W (ld nA); Tmp is nA x nA scratch.  Recursive halving, done level
// by level from the smallest blocks up: a node [lo, lo + 2s) with children
// [lo, mid) and [mid, mid + s) gets
//   W21 = -W22 (U21 W11)        (bufM holds U21 W11)
// All nodes of a level have the same size (the block count is padded to a
// power of two; nodes past the rank are empty), so a level is one batched
// FP64 launch per product when its products are small, and one batched
// tensor-core product per product (level_product) when they are large.
int tri_inverse(const Ctx& c, const double* U, double* W, double* Tmp) {
  const Plan& p = *c.p;
  const int64_t nA = p.nA, b = p.b;
  int64_t nb = 1;
  while (nb * b < nA) nb <<= 1;
  for (int64_t s = b; s < nb * b; s <<= 1) {
    const int64_t nodes = (nb * b) / (2 * s);
    const Dim rows = rdim(-s, s), cols = rdim(0, s);  // node 0: mid = s, lo = 0
    // nodes whose rows start inside the matrix (the others are empty)
    const int64_t live = nA > s ? (nA - s + 2 * s - 1) / (2 * s) : 0;
    if (prod_kind(p, S_PROD, live * s, s, s) == PK_EXACT && level_product_fits(p, s, live)) {
      // Tmp21 = U21 W11, then W21 = -W22 Tmp21
      CK(level_product(c, s, live, U + s * nA, rows, cols, W, cols, Tmp + s * nA, 1.0));
      CK(level_product(c, s, live, W + s * nA + s, rows, rows, Tmp + s * nA, cols, W + s * nA,
                       -1.0));
    } else if (prod_kind(p, S_PROD, s, s, s) == PK_FP64) {
      auto batched = [&](const double* A, const double* B, double* C, Dim M, Dim N, Dim K,
                         double alpha) -> cudaError_t {
        GemmParams g;
        std::memset(&g, 0, sizeof(g));
        g.A = A;
        g.B = B;
        g.C = C;
        g.lda = g.ldb = g.ldc = nA;
        g.M = M;
        g.N = N;
        g.K = K;
        g.alpha = alpha;
        g.beta = 0.0;
        g.rdev = c.rdev();
        // node z: lo = 2 s z, mid = lo + s (row and column offsets move by 2s)
        g.zA = g.zB = g.zC = 2 * s * nA + 2 * s;
        g.zM = g.zN = g.zK = (int32_t)(-2 * s);
        g.nz = (int32_t)nodes;
        KernelTimer t;
        t.gemm = &g;
        return t.run(KT_GEMM_FP64, c.s, [&] { return launch_dgemm(g, false, false, c.s); });
      };
      // Tmp = U21 W11:  (rows mid.., cols lo..)
      CK(batched(U + s * nA, W, Tmp + s * nA, rows, cols, cols, 1.0));
      // W21 = -W22 Tmp
      CK(batched(W + s * nA + s, Tmp + s * nA, W + s * nA, rows, cols, rows, -1.0));
    } else {
      for (int64_t z = 0; z < nodes; ++z) {
        const int64_t lo = 2 * s * z, mid = lo + s;
        if (mid >= nA) break;
        const Dim rz = rdim(-mid, s), cz = rdim(-lo, s);
        CK(matmul(c, S_PROD, U + mid * nA + lo, nA, false, W + lo * nA + lo, nA, false,
                  Tmp + mid * nA + lo, nA, rz, cz, cz, 1.0, 0.0, 0));
        CK(matmul(c, S_PROD, W + mid * nA + mid, nA, false, Tmp + mid * nA + lo, nA, false,
                  W + mid * nA + lo, nA, rz, cz, rz, -1.0, 0.0, 0));
      }
    }
  }
  return CPINV_OK;
}

// M = (L'L)^-1 into bufM (after front_rank with compaction).
int front_inverse(const Ctx& c) {
  const Plan& p = *c.p;
  const int64_t nA = p.nA;
  const int b = p.b;
  const Dim R = rdim(0, nA);
  // N = L'L (lower), into bufA
  CK(matmul(c, S_PROD, p.bufL, nA, true, p.bufL, nA, false, p.bufA, nA, R, R, hdim(nA), 1.0, 0.0,
            1));
  int rc = chol_exact_ok(p) ? factor_exact(c, p.bufA, nA, 1) : factor(c, p.bufA, nA, 1);
  if (rc) return rc;
  // W = U^-1: diagonal blocks from the factorisation, the rest by recursion
  CK(KernelTimer().run(KT_AUX, c.s, [&] {
    return launch_tri_inv_init(p.bufW, nA, nA, c.rdev(), p.Tinv, b, c.s);
  }));
  rc = tri_inverse(c, p.bufA, p.bufW, p.bufM);
  if (rc) return rc;
  // M = W'W: the lower triangle, mirrored (symmetric)
  CK(matmul(c, S_PROD, p.bufW, nA, true, p.bufW, nA, false, p.bufM, nA, R, R, R, 1.0, 0.0, 1));
  CK(KernelTimer().run(KT_AUX, c.s, [&] { return launch_mirror(p.bufM, nA, R, c.rdev(), c.s); }));
  return CPINV_OK;
}

// Reverse pass of W = G+ F (m >= n) with the kept-pivot set S fixed, after
// front_rank (with compaction) and front_inverse: L (n x r) in bufL, M =
// (L'L)^-1 in bufM, the mask in acc, the kept index of each pivot in colidx.
// Forward chain B = G'F, c1 = L'B, c2 = M c1, c3 = M c2, W = L c3, reversed:
//   Lbar = Wbar c3' + B cbar1',  cbar3 = L'Wbar,  Mbar = cbar3 c2' + cbar2 c1',
//   cbar2 = M cbar3,  cbar1 = M cbar2,  Bbar = L cbar1;
//   Nbar = -M Mbar M,  Lbar += L (Nbar + Nbar');
// the factor: Lbar masked to the factor's pattern (kept pivot c fills rows
// from its own index down), split into kept rows (L_S, lower triangular,
// L_S L_S' = A_SS) and rejected rows (L_D = A_DS L_S^-T on the pattern):
//   Abar_DS = Lbar_D X,  Lbar_S -= X' (Lbar_D' L_D),  X = L_S^-1,
//   Abar_SS = X' Phi(L_S' Lbar_S) X   (Phi: lower triangle, halved diagonal);
// and A = G'G, B = G'F:  Gbar = G (Abar + Abar') + F Bbar',  Fbar = G Bbar.
// Only the products with G or F (m rows) take the mode's tensor-core forms:
// the r x r factors of the reverse pass (L_S^-1, Mbar, Nbar) span many
// orders of magnitude within a row, where a fixed-point residue product of
// 53 bits per row loses the small entries that FP64 keeps.
int backward_body(const Ctx& c, const double* G, int64_t ldg, const double* F, int64_t ldf,
                  const double* dW, int64_t lddw, double* dG, int64_t lddg, double* dF,
                  int64_t lddf, double* W, int64_t ldw) {
  const Plan& p = *c.p;
  const int64_t n = p.n, m = p.m, k = p.k, nA = p.nA;
  const Dim R = rdim(0, nA), Nn = hdim(n), Kk = hdim(k), Dd = ddim(nA, nA);
  double* B = p.c1;                 // G'F        (n x k)
  double* c1 = p.c2;                // L'B        (r x k)
  double* c2 = p.c3;                // M c1
  double* c3 = p.e[0];              // M c2
  double *cb3 = p.e[1], *cb2 = p.e[2], *cb1 = p.e[3], *Bb = p.e[4];
  // forward chain, keeping its intermediates
  CK(matmul(c, S_CHAIN, G, ldg, true, F, ldf, false, B, k, Nn, Kk, hdim(m), 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, p.bufL, nA, true, B, k, false, c1, k, R, Kk, Nn, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, p.bufM, nA, false, c1, k, false, c2, k, R, Kk, R, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, p.bufM, nA, false, c2, k, false, c3, k, R, Kk, R, 1.0, 0.0, 0));
  if (W) CK(matmul(c, S_FP64, p.bufL, nA, false, c3, k, false, W, ldw, Nn, Kk, R, 1.0, 0.0, 0));
  // the chain, reversed
  CK(matmul(c, S_FP64, p.bufL, nA, true, dW, lddw, false, cb3, k, R, Kk, Nn, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, dW, lddw, false, c3, k, true, p.Lb, nA, Nn, R, Kk, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, cb3, k, false, c2, k, true, p.Mb, nA, R, R, Kk, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, p.bufM, nA, false, cb3, k, false, cb2, k, R, Kk, R, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, cb2, k, false, c1, k, true, p.Mb, nA, R, R, Kk, 1.0, 1.0, 0));
  CK(matmul(c, S_FP64, p.bufM, nA, false, cb2, k, false, cb1, k, R, Kk, R, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, B, k, false, cb1, k, true, p.Lb, nA, Nn, R, Kk, 1.0, 1.0, 0));
  CK(matmul(c, S_FP64, p.bufL, nA, false, cb1, k, false, Bb, k, Nn, Kk, R, 1.0, 0.0, 0));
  // Nbar = -M Mbar M  (S1 = Mbar M, bufA = Nbar);  Lbar += L Nbar + L Nbar'
  CK(matmul(c, S_FP64, p.Mb, nA, false, p.bufM, nA, false, p.S1, nA, R, R, R, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, p.bufM, nA, false, p.S1, nA, false, p.bufA, nA, R, R, R, -1.0, 0.0, 0));
  CK(matmul(c, S_FP64, p.bufL, nA, false, p.bufA, nA, false, p.Lb, nA, Nn, R, R, 1.0, 1.0, 0));
  CK(matmul(c, S_FP64, p.bufL, nA, false, p.bufA, nA, true, p.Lb, nA, Nn, R, R, 1.0, 1.0, 0));
  // the factor
  KernelTimer t;
  CK(t.run(KT_AUX, c.s,
           [&] { return launch_pivot_lists(p.acc, nA, p.pref, p.sidx, p.didx, c.s); }));
  CK(t.run(KT_AUX, c.s,
           [&] { return launch_pattern_mask(p.Lb, nA, nA, p.pref, c.rdev(), c.s); }));
  CK(t.run(KT_AUX, c.s, [&] {
    cudaError_t e = launch_gather_rows(p.bufL, nA, p.sidx, nA, 0, c.rdev(), p.LS, nA, c.s);
    if (e == cudaSuccess)
      e = launch_gather_rows(p.Lb, nA, p.sidx, nA, 0, c.rdev(), p.LbS, nA, c.s);
    if (e == cudaSuccess)
      e = launch_gather_rows(p.bufL, nA, p.didx, nA, 1, c.rdev(), p.LD, nA, c.s);
    if (e == cudaSuccess)
      e = launch_gather_rows(p.Lb, nA, p.didx, nA, 1, c.rdev(), p.LbD, nA, c.s);
    return e;
  }));
  // X = L_S^-1: inverted diagonal blocks, then the level-by-level recursion
  const int b = p.b <= 32 ? p.b : 32;
  CK(t.run(KT_AUX, c.s, [&] {
    return launch_tri_block_inverse(p.LS, nA, nA, c.rdev(), b, p.Tinv, c.s);
  }));
  CK(t.run(KT_AUX, c.s,
           [&] { return launch_tri_inv_init(p.X, nA, nA, c.rdev(), p.Tinv, b, c.s); }));
  {
    Plan q = p;
    q.b = b;
    q.mode = CPINV_MODE_FP64;  // see the note above on the r x r factors
    const Ctx cq{c.s, &q};
    if (int rc = tri_inverse(cq, p.LS, p.X, p.S1)) return rc;
  }
  // Abar_DS = Lbar_D X (into LD's place after its last use below: S2 first)
  CK(matmul(c, S_FP64, p.LbD, nA, true, p.LD, nA, false, p.S1, nA, R, R, Dd, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, p.X, nA, true, p.S1, nA, false, p.LbS, nA, R, R, R, -1.0, 1.0, 0));
  CK(matmul(c, S_FP64, p.LbD, nA, false, p.X, nA, false, p.LD, nA, Dd, R, R, 1.0, 0.0, 0));
  // Abar_SS = X' Phi(L_S' Lbar_S) X   (S1 = Phi(..), S2 = S1 X, LbD = X' S2)
  CK(matmul(c, S_FP64, p.LS, nA, true, p.LbS, nA, false, p.S1, nA, R, R, R, 1.0, 0.0, 0));
  CK(t.run(KT_AUX, c.s, [&] { return launch_phi(p.S1, nA, nA, c.rdev(), c.s); }));
  CK(matmul(c, S_FP64, p.S1, nA, false, p.X, nA, false, p.S2, nA, R, R, R, 1.0, 0.0, 0));
  CK(matmul(c, S_FP64, p.X, nA, true, p.S2, nA, false, p.LbD, nA, R, R, R, 1.0, 0.0, 0));
  // As = Abar + Abar' (n x n, into S1)
  CK(t.run(KT_AUX, c.s, [&] {
    return launch_sym_scatter(p.LbD, nA, p.LD, nA, p.colidx, p.pref, nA, p.S1, nA, c.s);
  }));
  // Gbar = G As + F Bbar',  Fbar = G Bbar
  CK(matmul(c, S_CHAIN, G, ldg, false, p.S1, nA, false, dG, lddg, hdim(m), Nn, Nn, 1.0, 0.0, 0));
  CK(matmul(c, S_CHAIN, F, ldf, false, Bb, k, true, dG, lddg, hdim(m), Nn, Kk, 1.0, 1.0, 0));
  if (dF)
    CK(matmul(c, S_CHAIN, G, ldg, false, Bb, k, false, dF, lddf, hdim(m), Kk, Nn, 1.0, 0.0, 0));
  return CPINV_OK;
}

// ---------------------------------------------------------------------------
// CUDA-graph replay of repeated calls.  Every launch of a call has a shape
// known on the host (the rank stays on the device), so a call is a fixed
// sequence of kernels for fixed arguments.  The first call with a given
// argument set runs directly; the second is captured on a library stream and
// instantiated; later ones replay the graph with one launch.  Off when
// tracing is on or CPINV_GRAPHS=0.
// ---------------------------------------------------------------------------
struct GraphKey {
  int32_t job, device, mode, panel;
  int64_t m, n, k, ld1, ld2, ld3, ld4, ld5, ld6;
  const void* p1;
  const void* p2;
  const void* p3;
  const void* p4;
  const void* p5;
  const void* p6;
  void* ws;
  size_t ws_bytes;
  double rel_tol;
};

struct GraphEntry {
  GraphKey key;
  int seen;
  int64_t launches;  // kernels in the captured sequence
  cudaGraphExec_t exec;
  uint64_t stamp;
};

struct GraphCache {
  std::mutex mu;
  std::vector<GraphEntry> entries;
  std::vector<std::pair<int, cudaStream_t>> side;
  uint64_t clock = 0;
};
GraphCache g_graphs;
constexpr size_t kMaxGraphs = 16;

thread_local int t_no_graph = 0;

bool graphs_enabled() {
  if (t_no_graph) return false;
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("CPINV_GRAPHS");
    on = (e && e[0] == '0') ? 0 : 1;
  }
  return on == 1 && !g_tr.on;
}

GraphKey make_key(int job, const Plan& p, int64_t ld1, int64_t ld2, int64_t ld3, const void* p1,
                  const void* p2, const void* p3, void* ws, size_t ws_bytes) {
  GraphKey k;
  std::memset(&k, 0, sizeof(k));
  k.job = job;
  cudaGetDevice(&k.device);
  k.mode = p.mode;
  k.panel = p.b;
  k.m = p.m;
  k.n = p.n;
  k.k = p.k;
  k.ld1 = ld1;
  k.ld2 = ld2;
  k.ld3 = ld3;
  k.p1 = p1;
  k.p2 = p2;
  k.p3 = p3;
  k.ws = ws;
  k.ws_bytes = ws_bytes;
  k.rel_tol = p.rel_tol;
  return k;
}

// Runs body(ctx) on `user` directly, or captured / replayed as a graph.
// keep_state: the call continues from the DevState a previous call left in
// the workspace (the reverse pass from a saved forward state), so it is not
// cleared.
template <class Body>
int run_pipeline(const Plan& p, cudaStream_t user, const GraphKey& key, Body&& body,
                 bool keep_state = false) {
  auto direct = [&]() -> int {
    Ctx c{user, &p};
    if (!keep_state) CK(cudaMemsetAsync(p.st, 0, sizeof(DevState), user));
    return body(c);
  };
  if (!graphs_enabled()) return direct();
  std::lock_guard<std::mutex> lock(g_graphs.mu);
  GraphEntry* e = nullptr;
  for (auto& x : g_graphs.entries)
    if (std::memcmp(&x.key, &key, sizeof(key)) == 0) e = &x;
  if (!e) {
    if (g_graphs.entries.size() >= kMaxGraphs) {
      size_t old = 0;
      for (size_t i = 1; i < g_graphs.entries.size(); ++i)
        if (g_graphs.entries[i].stamp < g_graphs.entries[old].stamp) old = i;
      if (g_graphs.entries[old].exec) cudaGraphExecDestroy(g_graphs.entries[old].exec);
      g_graphs.entries.erase(g_graphs.entries.begin() + (long)old);
    }
    GraphEntry ne;
    ne.key = key;
    ne.seen = 1;
    ne.launches = 0;
    ne.exec = nullptr;
    ne.stamp = ++g_graphs.clock;
    g_graphs.entries.push_back(ne);
    return direct();
  }
  e->stamp = ++g_graphs.clock;
  if (!e->exec) {
    cudaStream_t side = nullptr;
    for (auto& sd : g_graphs.side)
      if (sd.first == key.device) side = sd.second;
    if (!side) {
      CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
      g_graphs.side.push_back({key.device, side});
    }
    const int64_t l0 = g_launches.load();
    CK(cudaStreamBeginCapture(side, cudaStreamCaptureModeThreadLocal));
    Ctx c{side, &p};
    int rc = (keep_state || cudaMemsetAsync(p.st, 0, sizeof(DevState), side) == cudaSuccess)
                 ? body(c)
                 : CPINV_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(side, &graph);
    if (rc != CPINV_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc != CPINV_OK ? rc : CPINV_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return CPINV_ERR_CUDA;
    e->exec = exec;
    e->launches = g_launches.load() - l0;
    g_launches.fetch_sub(e->launches);  // counted again below, at launch
  }
  CK(cudaGraphLaunch(e->exec, user));
  g_launches.fetch_add(e->launches);
  return CPINV_OK;
}

}  // namespace

NoGraphScope::NoGraphScope() { ++t_no_graph; }
NoGraphScope::~NoGraphScope() { --t_no_graph; }
bool graph_replay_allowed() { return graphs_enabled(); }
void launches_add(int64_t n) { g_launches.fetch_add(n); }
cudaError_t trace_finish(cudaStream_t s, const int64_t* rdev) { return trace_resolve(s, rdev); }

namespace {

int finish(const Ctx& c, int64_t* rank_out) {
  CK(trace_resolve(c.s, c.rdev()));
  if (!rank_out) return CPINV_OK;
  DevState h;
  CK(cudaMemcpyAsync(&h, c.p->st, sizeof(DevState), cudaMemcpyDeviceToHost, c.s));
  CK(cudaStreamSynchronize(c.s));
  if (h.status & ST_NONFINITE) return CPINV_ERR_NONFINITE_INPUT;
  if (h.status & ST_NUMERICAL) return CPINV_ERR_NUMERICAL;
  if (h.status & ST_TIMEOUT) return CPINV_ERR_TIMEOUT;
  *rank_out = h.rank;
  return CPINV_OK;
}

int begin(Plan& p, Job job, void* ws, size_t ws_bytes) {
  if (!ws || ((uintptr_t)ws & 255u)) return CPINV_ERR_WORKSPACE;
  if (ws_bytes < plan_bytes(p, job)) return CPINV_ERR_WORKSPACE;
  Arena a{(char*)ws, 0};
  carve(p, a, job);
  return CPINV_OK;
}

}  // namespace
}  // namespace cpinv

using namespace cpinv;

namespace {

// C = alpha op(A) op(B) + beta C in the given arithmetic (lower: only the
// lower triangle of a square C); the body of cpinv_matmul.
int product_raw(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K, double alpha,
                const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                int64_t ldc, int32_t mode, int32_t bits, int lower, void* workspace,
                size_t workspace_bytes, int32_t check, void* stream) {
  if (M < 0 || N < 0 || K < 0) return CPINV_ERR_INVALID_ARG;
  if (mode != CPINV_MODE_FP64 && mode != CPINV_MODE_EXACT_SLICE &&
      mode != CPINV_MODE_SPLIT_BF16X3)
    return CPINV_ERR_INVALID_ARG;
  const int64_t arows = transA ? K : M, acols = transA ? M : K;
  const int64_t brows = transB ? N : K, bcols = transB ? K : N;
  if ((arows > 0 && lda < acols) || (brows > 0 && ldb < bcols) || ldc < N)
    return CPINV_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return CPINV_OK;
  if (!C || (K > 0 && (!A || !B))) return CPINV_ERR_INVALID_ARG;
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return CPINV_ERR_INVALID_ARG;
  if (C == A || C == B) return CPINV_ERR_INVALID_ARG;  // C must not alias an operand
  const int beta_bits = bits ? bits : 53;
  if (mode == CPINV_MODE_EXACT_SLICE && (beta_bits < 1 || beta_bits > 62)) return CPINV_ERR_INVALID_ARG;
  const bool same = A == B && lda == ldb && (transA != 0) != (transB != 0) && M == N;
  size_t need = 0;
  if (mode == CPINV_MODE_FP64) need = 256;
  else if (mode == CPINV_MODE_SPLIT_BF16X3) need = 1024 + split_workspace_bytes(M, N, K, same);
  else {
    const int64_t Kc = K < kCrtMaxK ? (K > 0 ? K : 1) : kCrtMaxK;
    const int nm = crt_moduli_for(Kc, beta_bits, beta_bits);
    if (nm < 0) return CPINV_ERR_INVALID_ARG;
    need = 1024 + crt_workspace_bytes(M, N, Kc, nm, same);
  }
  if (!workspace || ((uintptr_t)workspace & 255u) || workspace_bytes < need)
    return CPINV_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = (DevState*)workspace;
  CK(cudaMemsetAsync(st, 0, sizeof(DevState), s));
  GemmParams g;
  std::memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.C = C;
  g.lda = lda;
  g.ldb = ldb;
  g.ldc = ldc;
  g.M = hdim(M);
  g.N = hdim(N);
  g.K = hdim(K);
  g.alpha = alpha;
  g.beta = beta;
  g.rdev = &st->rank;
  g.lower = lower && M == N;
  if (mode == CPINV_MODE_FP64 || K == 0) {
    KernelTimer t;
    t.gemm = &g;
    CK(t.run(KT_GEMM_FP64, s, [&] { return launch_dgemm(g, transA != 0, transB != 0, s); }));
  } else if (mode == CPINV_MODE_SPLIT_BF16X3) {
    CrtGemm sg;
    sg.p = g;
    sg.transA = transA != 0;
    sg.transB = transB != 0;
    sg.same_operand = same;
    sg.betaA = sg.betaB = 0;
    sg.ws = (char*)workspace + 1024;
    sg.ws_bytes = workspace_bytes - 1024;
    sg.st = st;
    KernelTimer t;
    CK(launch_split_gemm(sg, s, &t));
  } else {
    CK(crt_product(g, transA != 0, transB != 0, beta_bits, same, (char*)workspace + 1024,
                   workspace_bytes - 1024, st, s));
  }
  CK(trace_resolve(s, &st->rank));
  if (!check) return CPINV_OK;
  DevState h;
  CK(cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h.status & ST_NONFINITE) return CPINV_ERR_NONFINITE_INPUT;
  if (h.status & ST_TIMEOUT) return CPINV_ERR_TIMEOUT;
  return CPINV_OK;
}

}  // namespace

extern "C" {

void cpinv_default_opts(cpinv_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = CPINV_MODE_FP64;
  o->slices = 0;
  o->panel = 0;
  o->rel_tol = 1e-9;
}

const char* cpinv_status_string(int status) {
  switch (status) {
    case CPINV_OK: return "ok";
    case CPINV_ERR_INVALID_ARG: return "invalid argument";
    case CPINV_ERR_NONFINITE_INPUT: return "non-finite input";
    case CPINV_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case CPINV_ERR_CUDA: return "CUDA error";
    case CPINV_ERR_NUMERICAL: return "L'L not positive definite in FP64";
    case CPINV_ERR_UNSUPPORTED: return "unsupported mode or size";
    case CPINV_ERR_TIMEOUT: return "a device-side wait timed out";
    default: return "unknown status";
  }
}

int cpinv_version(void) { return 100; }

size_t cpinv_rank_workspace_size(int64_t m, int64_t n, const cpinv_opts* o) {
  Plan p{};
  if (m < 0 || n < 0 || !make_plan(p, m, n, 0, o)) return 0;
  return plan_bytes(p, JOB_RANK);
}

size_t cpinv_pinv_workspace_size(int64_t m, int64_t n, const cpinv_opts* o) {
  Plan p{};
  if (m < 0 || n < 0 || !make_plan(p, m, n, 0, o)) return 0;
  return plan_bytes(p, JOB_PINV);
}

size_t cpinv_lstsq_workspace_size(int64_t m, int64_t n, int64_t k, const cpinv_opts* o) {
  Plan p{};
  if (m < 0 || n < 0 || k < 0 || !make_plan(p, m, n, k, o)) return 0;
  return plan_bytes(p, JOB_LSTSQ);
}

static int check_opts(const cpinv_opts* o) {
  if (!o) return CPINV_OK;
  if (o->mode != CPINV_MODE_FP64 && o->mode != CPINV_MODE_EXACT_SLICE &&
      o->mode != CPINV_MODE_SPLIT_BF16X3)
    return CPINV_ERR_INVALID_ARG;
  if (o->panel < 0 || o->panel > 32 || (o->panel && 64 % o->panel) || o->reserved != 0)
    return CPINV_ERR_INVALID_ARG;
  if (!(o->rel_tol >= 0.0) || !std::isfinite(o->rel_tol)) return CPINV_ERR_INVALID_ARG;
  return CPINV_OK;
}

int cpinv_rank(const double* G, int64_t m, int64_t n, int64_t ldg, uint8_t* accepted_out,
               void* workspace, size_t workspace_bytes, const cpinv_opts* o, int64_t* rank_out,
               void* stream) {
  if (rank_out) *rank_out = -1;
  if (int rc = check_opts(o)) return rc;
  if (m < 0 || n < 0 || ldg < n) return CPINV_ERR_INVALID_ARG;
  if (m == 0 || n == 0) {
    if (rank_out) *rank_out = 0;
    return CPINV_OK;
  }
  if (!G) return CPINV_ERR_INVALID_ARG;
  Plan p{};
  if (!make_plan(p, m, n, 0, o)) return CPINV_ERR_INVALID_ARG;
  if (int rc = begin(p, JOB_RANK, workspace, workspace_bytes)) return rc;
  cudaStream_t us = (cudaStream_t)stream;
  const GraphKey key = make_key(JOB_RANK, p, ldg, 0, 0, G, accepted_out, nullptr, workspace,
                                workspace_bytes);
  int rc = run_pipeline(p, us, key, [&](const Ctx& c) -> int {
    if (int r = front_rank(c, G, ldg, false)) return r;
    if (accepted_out)
      CK(KernelTimer().run(KT_AUX, c.s,
                           [&] { return launch_copy_mask(p.acc, accepted_out, p.nA, c.s); }));
    return CPINV_OK;
  });
  if (rc) return rc;
  return finish(Ctx{us, &p}, rank_out);
}

int cpinv_pinv(const double* G, int64_t m, int64_t n, int64_t ldg, double* Gp, int64_t ldgp,
               void* workspace, size_t workspace_bytes, const cpinv_opts* o, int64_t* rank_out,
               void* stream) {
  if (rank_out) *rank_out = -1;
  if (int rc = check_opts(o)) return rc;
  if (m < 0 || n < 0 || ldg < n || ldgp < m) return CPINV_ERR_INVALID_ARG;
  if (m == 0 || n == 0) {
    if (rank_out) *rank_out = 0;
    return CPINV_OK;
  }
  if (!G || !Gp) return CPINV_ERR_INVALID_ARG;
  Plan p{};
  if (!make_plan(p, m, n, 0, o)) return CPINV_ERR_INVALID_ARG;
  if (int rc = begin(p, JOB_PINV, workspace, workspace_bytes)) return rc;
  cudaStream_t us = (cudaStream_t)stream;
  const GraphKey key = make_key(JOB_PINV, p, ldg, ldgp, 0, G, Gp, nullptr, workspace,
                                workspace_bytes);
  int rc = run_pipeline(p, us, key, [&](const Ctx& c) -> int {
    if (int r = front_rank(c, G, ldg, true)) return r;
    if (int r = front_inverse(c)) return r;
    const int64_t nA = p.nA;
    const Dim R = rdim(0, nA);
    // X = L M  (bufW),  K = X X'  (bufA: the lower triangle, mirrored)
    CK(matmul(c, S_CHAIN, p.bufL, nA, false, p.bufM, nA, false, p.bufW, nA, hdim(nA), R, R, 1.0,
              0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufW, nA, false, p.bufW, nA, true, p.bufA, nA, hdim(nA), hdim(nA), R,
              1.0, 0.0, 1));
    CK(KernelTimer().run(KT_AUX, c.s,
                         [&] { return launch_mirror(p.bufA, nA, hdim(nA), c.rdev(), c.s); }));
    if (!p.trans)  // G+ = K G'   (n x n)(n x m)
      CK(matmul(c, S_CHAIN, p.bufA, nA, false, G, ldg, true, Gp, ldgp, hdim(n), hdim(m), hdim(n),
                1.0, 0.0, 0));
    else  // G+ = G' K   (n x m)(m x m)
      CK(matmul(c, S_CHAIN, G, ldg, true, p.bufA, nA, false, Gp, ldgp, hdim(n), hdim(m), hdim(m),
                1.0, 0.0, 0));
    return CPINV_OK;
  });
  if (rc) return rc;
  return finish(Ctx{us, &p}, rank_out);
}

int cpinv_lstsq(const double* G, int64_t m, int64_t n, int64_t ldg, const double* F, int64_t k,
                int64_t ldf, double* W, int64_t ldw, void* workspace, size_t workspace_bytes,
                const cpinv_opts* o, int64_t* rank_out, void* stream) {
  if (rank_out) *rank_out = -1;
  if (int rc = check_opts(o)) return rc;
  if (m < 0 || n < 0 || k < 0 || ldg < n || ldf < k || ldw < k) return CPINV_ERR_INVALID_ARG;
  if (m == 0 || n == 0 || k == 0) {
    // W (n x k) = 0 when m == 0; nothing to write when n == 0 or k == 0.
    if (m == 0 && n > 0 && k > 0) {
      if (!W) return CPINV_ERR_INVALID_ARG;
      CK(cudaMemset2DAsync(W, (size_t)ldw * sizeof(double), 0, (size_t)k * sizeof(double),
                           (size_t)n, (cudaStream_t)stream));
    }
    if (rank_out && (m == 0 || n == 0)) *rank_out = 0;
    if (k == 0 && m > 0 && n > 0 && rank_out) {
      // rank still defined: run the rank query path
      return cpinv_rank(G, m, n, ldg, nullptr, workspace, workspace_bytes, o, rank_out, stream);
    }
    return CPINV_OK;
  }
  if (!G || !F || !W) return CPINV_ERR_INVALID_ARG;
  Plan p{};
  if (!make_plan(p, m, n, k, o)) return CPINV_ERR_INVALID_ARG;
  if (int rc = begin(p, JOB_LSTSQ, workspace, workspace_bytes)) return rc;
  cudaStream_t us = (cudaStream_t)stream;
  const GraphKey key = make_key(JOB_LSTSQ, p, ldg, ldf, ldw, G, F, W, workspace,
                                workspace_bytes);
  int rc = run_pipeline(p, us, key, [&](const Ctx& c) -> int {
    if (int r = front_rank(c, G, ldg, true)) return r;
    if (int r = front_inverse(c)) return r;
    const int64_t nA = p.nA;
    const Dim R = rdim(0, nA);
    if (!p.trans) {
      // c1 <- G'F (n x k);  c2 <- L' c1 (r x k)
      CK(matmul(c, S_CHAIN, G, ldg, true, F, ldf, false, p.c1, k, hdim(n), hdim(k), hdim(m), 1.0,
                0.0, 0));
      CK(matmul(c, S_CHAIN, p.bufL, nA, true, p.c1, k, false, p.c2, k, R, hdim(k), hdim(nA), 1.0, 0.0,
                0));
    } else {
      // c2 <- L' F (r x k)
      CK(matmul(c, S_CHAIN, p.bufL, nA, true, F, ldf, false, p.c2, k, R, hdim(k), hdim(nA), 1.0, 0.0,
                0));
    }
    CK(matmul(c, S_CHAIN, p.bufM, nA, false, p.c2, k, false, p.c3, k, R, hdim(k), R, 1.0, 0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufM, nA, false, p.c3, k, false, p.c2, k, R, hdim(k), R, 1.0, 0.0, 0));
    if (!p.trans) {
      CK(matmul(c, S_CHAIN, p.bufL, nA, false, p.c2, k, false, W, ldw, hdim(n), hdim(k), R, 1.0, 0.0,
                0));
    } else {
      // t = L c (m x k) into c1, W = G' t
      CK(matmul(c, S_CHAIN, p.bufL, nA, false, p.c2, k, false, p.c1, k, hdim(m), hdim(k), R, 1.0,
                0.0, 0));
      CK(matmul(c, S_CHAIN, G, ldg, true, p.c1, k, false, W, ldw, hdim(n), hdim(k), hdim(m), 1.0, 0.0,
                0));
    }
    return CPINV_OK;
  });
  if (rc) return rc;
  return finish(Ctx{us, &p}, rank_out);
}

size_t cpinv_lstsq_gram_workspace_size(int64_t n, int64_t k, const cpinv_opts* o) {
  Plan p{};
  if (n < 0 || k < 0 || !make_plan(p, n, n, k > 0 ? k : 1, o)) return 0;
  return plan_bytes(p, JOB_LSTSQ);
}

int cpinv_lstsq_gram(const double* A, int64_t n, int64_t lda, const double* B, int64_t k,
                     int64_t ldb, double* W, int64_t ldw, void* workspace, size_t workspace_bytes,
                     const cpinv_opts* o, int64_t* rank_out, void* stream) {
  if (rank_out) *rank_out = -1;
  if (int rc = check_opts(o)) return rc;
  if (n < 0 || k < 0 || lda < n || ldb < k || ldw < k) return CPINV_ERR_INVALID_ARG;
  if (n == 0) {
    if (rank_out) *rank_out = 0;
    return CPINV_OK;
  }
  // k == 0 still factors A: the rank is reported, no W is written
  if (!A || (k > 0 && (!B || !W))) return CPINV_ERR_INVALID_ARG;
  Plan p{};
  if (!make_plan(p, n, n, k > 0 ? k : 1, o)) return CPINV_ERR_INVALID_ARG;
  if (int rc = begin(p, JOB_LSTSQ, workspace, workspace_bytes)) return rc;
  cudaStream_t us = (cudaStream_t)stream;
  const GraphKey key = make_key(JOB_GRAM_LSTSQ, p, lda, ldb, ldw, A, B, W, workspace,
                                workspace_bytes);
  int rc = run_pipeline(p, us, key, [&](const Ctx& c) -> int {
    // the caller's Gram matrix (lower triangle read) into the factor buffer
    CK(cudaMemcpy2DAsync(p.bufA, (size_t)n * sizeof(double), A, (size_t)lda * sizeof(double),
                         (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice, c.s));
    if (int r = rank_from_gram(c, true)) return r;
    if (k == 0) return CPINV_OK;
    if (int r = front_inverse(c)) return r;
    const int64_t nA = p.nA;
    const Dim R = rdim(0, nA);
    // W = L (M (M (L' B)))
    CK(matmul(c, S_CHAIN, p.bufL, nA, true, B, ldb, false, p.c2, k, R, hdim(k), hdim(nA), 1.0,
              0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufM, nA, false, p.c2, k, false, p.c3, k, R, hdim(k), R, 1.0, 0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufM, nA, false, p.c3, k, false, p.c2, k, R, hdim(k), R, 1.0, 0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufL, nA, false, p.c2, k, false, W, ldw, hdim(nA), hdim(k), R, 1.0,
              0.0, 0));
    return CPINV_OK;
  });
  if (rc) return rc;
  return finish(Ctx{us, &p}, rank_out);
}

size_t cpinv_lstsq_backward_workspace_size(int64_t m, int64_t n, int64_t k, const cpinv_opts* o) {
  Plan p{};
  if (m < 0 || n < 0 || k < 0 || !make_plan(p, m, n, k, o)) return 0;
  return plan_bytes(p, JOB_BACKWARD);
}

int cpinv_lstsq_backward(const double* G, int64_t m, int64_t n, int64_t ldg, const double* F,
                         int64_t k, int64_t ldf, const double* dW, int64_t lddw, double* dG,
                         int64_t lddg, double* dF, int64_t lddf, double* W, int64_t ldw,
                         void* workspace, size_t workspace_bytes, const cpinv_opts* o,
                         int64_t* rank_out, void* stream) {
  if (rank_out) *rank_out = -1;
  if (int rc = check_opts(o)) return rc;
  if (m < 0 || n < 0 || k < 0 || ldg < n || ldf < k || lddw < k || lddg < n ||
      (dF && lddf < k) || (W && ldw < k))
    return CPINV_ERR_INVALID_ARG;
  if (m < n) return CPINV_ERR_UNSUPPORTED;
  cudaStream_t us = (cudaStream_t)stream;
  if (m == 0 || n == 0 || k == 0) {
    // W = 0 and both adjoints vanish
    if (n > 0 && m > 0) {
      if (!dG) return CPINV_ERR_INVALID_ARG;
      CK(cudaMemset2DAsync(dG, (size_t)lddg * sizeof(double), 0, (size_t)n * sizeof(double),
                           (size_t)m, us));
    }
    if (rank_out) *rank_out = 0;
    if (k == 0 && m > 0 && n > 0 && rank_out)
      return cpinv_rank(G, m, n, ldg, nullptr, workspace, workspace_bytes, o, rank_out, stream);
    return CPINV_OK;
  }
  if (!G || !F || !dW || !dG) return CPINV_ERR_INVALID_ARG;
  Plan p{};
  if (!make_plan(p, m, n, k, o)) return CPINV_ERR_INVALID_ARG;
  if (int rc = begin(p, JOB_BACKWARD, workspace, workspace_bytes)) return rc;
  GraphKey key = make_key(JOB_BACKWARD, p, ldg, ldf, lddw, G, F, dW, workspace, workspace_bytes);
  key.ld4 = lddg;
  key.ld5 = dF ? lddf : 0;
  key.ld6 = W ? ldw : 0;
  key.p4 = dG;
  key.p5 = dF;
  key.p6 = W;
  int rc = run_pipeline(p, us, key, [&](const Ctx& c) -> int {
    if (int r = front_rank(c, G, ldg, true)) return r;
    if (int r = front_inverse(c)) return r;
    return backward_body(c, G, ldg, F, ldf, dW, lddw, dG, lddg, dF, lddf, W, ldw);
  });
  if (rc) return rc;
  return finish(Ctx{us, &p}, rank_out);
}

size_t cpinv_lstsq_state_size(int64_t m, int64_t n, int64_t k, const cpinv_opts* o) {
  return cpinv_lstsq_backward_workspace_size(m, n, k, o);
}

int cpinv_lstsq_forward(const double* G, int64_t m, int64_t n, int64_t ldg, const double* F,
                        int64_t k, int64_t ldf, double* W, int64_t ldw, void* state,
                        size_t state_bytes, const cpinv_opts* o, int64_t* rank_out,
                        void* stream) {
  if (rank_out) *rank_out = -1;
  if (int rc = check_opts(o)) return rc;
  if (m < 0 || n < 0 || k < 0 || ldg < n || ldf < k || ldw < k) return CPINV_ERR_INVALID_ARG;
  if (m < n) return CPINV_ERR_UNSUPPORTED;
  if (m == 0 || n == 0 || k == 0) return CPINV_ERR_UNSUPPORTED;  // nothing to differentiate
  if (!G || !F || !W) return CPINV_ERR_INVALID_ARG;
  Plan p{};
  if (!make_plan(p, m, n, k, o)) return CPINV_ERR_INVALID_ARG;
  if (int rc = begin(p, JOB_BACKWARD, state, state_bytes)) return rc;
  cudaStream_t us = (cudaStream_t)stream;
  const GraphKey key = make_key(JOB_FORWARD_SAVE, p, ldg, ldf, ldw, G, F, W, state, state_bytes);
  int rc = run_pipeline(p, us, key, [&](const Ctx& c) -> int {
    if (int r = front_rank(c, G, ldg, true)) return r;
    if (int r = front_inverse(c)) return r;
    const int64_t nA = p.nA;
    const Dim R = rdim(0, nA);
    // W = L (M (M (L' (G'F)))), as cpinv_lstsq (m >= n)
    CK(matmul(c, S_CHAIN, G, ldg, true, F, ldf, false, p.c1, k, hdim(n), hdim(k), hdim(m), 1.0,
              0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufL, nA, true, p.c1, k, false, p.c2, k, R, hdim(k), hdim(nA), 1.0,
              0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufM, nA, false, p.c2, k, false, p.c3, k, R, hdim(k), R, 1.0, 0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufM, nA, false, p.c3, k, false, p.c2, k, R, hdim(k), R, 1.0, 0.0, 0));
    CK(matmul(c, S_CHAIN, p.bufL, nA, false, p.c2, k, false, W, ldw, hdim(n), hdim(k), R, 1.0, 0.0,
              0));
    return CPINV_OK;
  });
  if (rc) return rc;
  return finish(Ctx{us, &p}, rank_out);
}

int cpinv_lstsq_backward_from_state(const double* G, int64_t m, int64_t n, int64_t ldg,
                                    const double* F, int64_t k, int64_t ldf, const double* dW,
                                    int64_t lddw, double* dG, int64_t lddg, double* dF,
                                    int64_t lddf, void* state, size_t state_bytes,
                                    const cpinv_opts* o, int64_t* rank_out, void* stream) {
  if (rank_out) *rank_out = -1;
  if (int rc = check_opts(o)) return rc;
  if (m < 0 || n < 0 || k < 0 || ldg < n || ldf < k || lddw < k || lddg < n ||
      (dF && lddf < k))
    return CPINV_ERR_INVALID_ARG;
  if (m < n || m == 0 || n == 0 || k == 0) return CPINV_ERR_UNSUPPORTED;
  if (!G || !F || !dW || !dG) return CPINV_ERR_INVALID_ARG;
  Plan p{};
  if (!make_plan(p, m, n, k, o)) return CPINV_ERR_INVALID_ARG;
  if (int rc = begin(p, JOB_BACKWARD, state, state_bytes)) return rc;
  cudaStream_t us = (cudaStream_t)stream;
  GraphKey key = make_key(JOB_BACKWARD_STATE, p, ldg, ldf, lddw, G, F, dW, state, state_bytes);
  key.ld4 = lddg;
  key.ld5 = dF ? lddf : 0;
  key.p4 = dG;
  key.p5 = dF;
  // L, M, the kept mask, the kept index of each pivot and the rank are the
  // forward call's, in the state: only the reverse pass runs
  int rc = run_pipeline(
      p, us, key,
      [&](const Ctx& c) -> int {
        return backward_body(c, G, ldg, F, ldf, dW, lddw, dG, lddg, dF, lddf, nullptr, 0);
      },
      /*keep_state=*/true);
  if (rc) return rc;
  return finish(Ctx{us, &p}, rank_out);
}

size_t cpinv_matmul_workspace_size(int64_t M, int64_t N, int64_t K, int32_t mode, int32_t bits,
                                   int32_t symmetric) {
  if (M < 0 || N < 0 || K < 0) return 0;
  if (mode == CPINV_MODE_FP64) return 256;
  if (mode == CPINV_MODE_SPLIT_BF16X3) return 1024 + split_workspace_bytes(M, N, K, symmetric != 0);
  if (mode != CPINV_MODE_EXACT_SLICE) return 0;
  const int beta = bits ? bits : 53;
  if (beta < 1 || beta > 62) return 0;
  const int64_t Kc = K < kCrtMaxK ? (K > 0 ? K : 1) : kCrtMaxK;
  const int nm = crt_moduli_for(Kc, beta, beta);
  if (nm < 0) return 0;
  return 1024 + crt_workspace_bytes(M, N, Kc, nm, symmetric != 0);
}

int cpinv_matmul(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                 int64_t ldc, int32_t mode, int32_t bits, void* workspace, size_t workspace_bytes,
                 int32_t check, void* stream) {
  return product_raw(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, mode, bits, 0,
                     workspace, workspace_bytes, check, stream);
}

size_t cpinv_gram_update_workspace_size(int64_t m, int64_t n, int64_t k, int32_t mode) {
  if (m < 0 || n < 0 || k < 0) return 0;
  const size_t a = cpinv_matmul_workspace_size(n, n, m, mode, 62, 1);
  const size_t b = cpinv_matmul_workspace_size(n, k, m, mode, 53, 0);
  if (!a || !b) return 0;
  return a > b ? a : b;
}

int cpinv_gram_update(const double* G, int64_t m, int64_t n, int64_t ldg, const double* F,
                      int64_t k, int64_t ldf, double* A, int64_t lda, double* B, int64_t ldb,
                      int32_t mode, void* workspace, size_t workspace_bytes, void* stream) {
  if (m < 0 || n < 0 || k < 0 || lda < n || (F && (ldf < k || !B || ldb < k))) return CPINV_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return CPINV_OK;
  if (!G || !A || ldg < n) return CPINV_ERR_INVALID_ARG;
  // A (lower) += G'G: the Gram increment in the arithmetic of the Gram (62-bit
  // integers in the exact-slice mode: each increment correctly rounded)
  int rc = product_raw(1, 0, n, n, m, 1.0, G, ldg, G, ldg, 1.0, A, lda, mode, 62, 1, workspace,
                       workspace_bytes, 0, stream);
  if (rc || !F || k == 0) return rc;
  return product_raw(1, 0, n, k, m, 1.0, G, ldg, F, ldf, 1.0, B, ldb, mode, 53, 0, workspace,
                     workspace_bytes, 0, stream);
}

int cpinv_selftest_wait_timeout(void* workspace, size_t workspace_bytes, void* stream) {
  if (!workspace || workspace_bytes < sizeof(DevState)) return CPINV_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = (DevState*)workspace;
  if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) return CPINV_ERR_CUDA;
  if (launch_wait_selftest(st, s) != cudaSuccess) return CPINV_ERR_CUDA;
  DevState h;
  if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CPINV_ERR_CUDA;
  return (h.status & ST_TIMEOUT) ? CPINV_ERR_TIMEOUT : CPINV_OK;
}

int cpinv_profile_enable(int on) {
  const int prev = g_tr.on ? 1 : 0;
  for (auto& t : g_tr.recs) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  g_tr.recs.clear();
  g_tr.on = on != 0;
  return prev;
}

int cpinv_profile_read(cpinv_profile_entry* out, int max_entries) {
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;
  int64_t launches[KT_COUNT] = {0};
  double ms[KT_COUNT] = {0}, flops[KT_COUNT] = {0};
  for (auto& t : g_tr.recs) {
    float e = 0.f;
    if (cudaEventElapsedTime(&e, t.e0, t.e1) != cudaSuccess) return -1;
    launches[t.kind] += 1;
    ms[t.kind] += e;
    flops[t.kind] += t.resolved ? t.flops : 0.0;
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  g_tr.recs.clear();
  int n = 0;
  for (int k = 0; k < KT_COUNT; ++k) {
    if (!launches[k]) continue;
    if (out && n < max_entries) {
      std::memset(&out[n], 0, sizeof(out[n]));
      std::strncpy(out[n].name, kKindName[k], sizeof(out[n].name) - 1);
      out[n].launches = launches[k];
      out[n].ms = ms[k];
      out[n].flops = flops[k];
    }
    ++n;
  }
  return n;
}

int cpinv_profile_timeline(cpinv_timeline_entry* out, int max_entries) {
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;
  if (g_tr.recs.empty()) return 0;
  const cudaEvent_t origin = g_tr.recs.front().e0;
  int n = 0;
  for (auto& t : g_tr.recs) {
    if (out && n < max_entries) {
      float a = 0.f, b = 0.f;
      if (cudaEventElapsedTime(&a, origin, t.e0) != cudaSuccess ||
          cudaEventElapsedTime(&b, origin, t.e1) != cudaSuccess)
        return -1;
      std::memset(&out[n], 0, sizeof(out[n]));
      std::strncpy(out[n].name, kKindName[t.kind], sizeof(out[n].name) - 1);
      out[n].start_ms = a;
      out[n].end_ms = b;
    }
    ++n;
  }
  return n;
}

int64_t cpinv_launch_count(void) { return g_launches.load(); }

}  // extern "C"
