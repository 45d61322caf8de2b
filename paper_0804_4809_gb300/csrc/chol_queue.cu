// Full-rank Cholesky of every problem of a batch in ONE persistent launch
// that pulls its work from a device queue (the batched path's factorisations,
// Appendix of the paper, natural order, strict test d > tol).
//
// Work is cut into tasks on 32 x 32 tiles of each problem's matrix (panel
// width 32, right-looking):
//   DIAG(z, p)        factor diagonal block p (pivot tests, four warps)
//   SOLVE(z, p, i)    block row i > p of panel p: forward substitution
//                     against the factored block
//   UPD(z, p, i, j)   tile (i, j), p < j <= i:  A_ij -= L_ip L_jp'
// The host lists the tasks in an order where every task comes after the
// ones it depends on (panel by panel; in a panel DIAG, then SOLVE, then UPD);
// CTAs claim them in that order with an atomic counter.  A claimed task
// waits (bounded) for its inputs, flagged per problem by tile versions:
//   ver[i][j]   panels applied to tile (i, j) (UPD of panel p needs p, sets p + 1)
//   solved[i]   panels solved in block row i (SOLVE of panel p sets p + 1)
//   diag[p]     1 once block p is factored
// Every task a CTA waits for was claimed earlier by a CTA that is running,
// so the wait ends whatever the number of resident CTAs; a wait that runs
// out (about a second) records ST_TIMEOUT and raises the launch's abort
// flag, after which every CTA stops claiming and exits.
#include <cstdint>
#include <cstring>

#include "chol_device.cuh"
#include "common.cuh"
#include "kernels.h"

namespace cpinv {
namespace {

constexpr int kQThreads = chol::kDiagThreads;  // 128: four warps
constexpr uint32_t kQSpinLimit = 1u << 22;

__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int32_t v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: bounded wait until every (flag >= want) holds; false on expiry or
// when the launch aborted (then the abort flag is set for everyone).
__device__ bool wait_flags(const int32_t* const* f, const int32_t* want, int nf, int32_t* abort,
                           int32_t* status) {
  for (uint32_t it = 0; it < kQSpinLimit; ++it) {
    bool ok = true;
    for (int q = 0; q < nf; ++q) ok = ok && ld_acquire(f[q]) >= want[q];
    if (ok) return true;
    if (ld_acquire(abort)) return false;
    __nanosleep(it < 32 ? 64 : 512);
  }
  atomicOr(status, ST_TIMEOUT);
  atomicExch(abort, 1);
  return false;
}

struct Tile {
  double a[32][33];
  double b[32][33];
};

__global__ void __launch_bounds__(kQThreads) chol_queue_kernel(QueueFactor q) {
  __shared__ union {
    chol::DiagScratch diag;
    Tile t;
  } sm;
  __shared__ int s_task, s_go;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* head = q.head;
  int32_t* abort = q.head + 1;
  for (;;) {
    if (tid == 0) s_task = ld_acquire(abort) ? q.ntasks : atomicAdd(head, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= q.ntasks) break;
    const QueueTask tk = q.tasks[t];
    const int z = tk.z, p = tk.p, i = tk.i, j = tk.j;
    double* A = q.A + (int64_t)z * q.zA;
    const int64_t ld = q.np;
    DevState* st = q.st + z;
    const int64_t* rdev = &st->rank;
    const Dim nd{0, q.np, q.sel, 0};
    const int64_t n = eval_dim(nd, rdev);
    const int nbq = q.nb_max;
    int32_t* fl = q.flags + (int64_t)z * q.zFlags;
    int32_t* ver = fl;                        // [nb][nb]
    int32_t* solved = fl + nbq * nbq;         // [nb]
    int32_t* diag = solved + nbq;             // [nb]
    // inputs
    if (tid == 0) {
      const int32_t* f[3];
      int32_t w[3];
      int nf = 0;
      if (tk.kind == kQDiag) {
        f[nf] = ver + p * nbq + p; w[nf++] = p;
      } else if (tk.kind == kQSolve) {
        f[nf] = diag + p; w[nf++] = 1;
        f[nf] = ver + i * nbq + p; w[nf++] = p;
      } else {
        f[nf] = solved + i; w[nf++] = p + 1;
        f[nf] = solved + j; w[nf++] = p + 1;
        f[nf] = ver + i * nbq + j; w[nf++] = p;
      }
      s_go = wait_flags(f, w, nf, abort, &st->status) ? 1 : 0;
    }
    __syncthreads();
    if (!s_go) continue;  // aborted: the next claim sees the flag and exits
    const int64_t k0 = 32 * (int64_t)p;
    if (tk.kind == kQDiag) {
      chol::diag_chol_block(A, ld, nd, k0, 32, st, rdev, q.spd ? nullptr : q.acc + (int64_t)z * q.zAcc,
                            q.dinv + (int64_t)z * q.zDinv + k0, q.spd, sm.diag);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(diag + p, 1);
      }
    } else if (tk.kind == kQSolve) {
      // rows 32 i .. of panel p: L(r, P) T' = A(r, P), T the factored block;
      // Ts[r][c] = T(r, c) / T(c, c), one warp per row, lane c = column c
      const double* dv = q.dinv + (int64_t)z * q.zDinv + k0;
      const int bw = (int)((n - k0) < 32 ? (n - k0) : 32);
      for (int e = tid; e < 32 * 32; e += kQThreads) {
        const int r = e >> 5, c = e & 31;
        sm.t.a[r][c] = (bw > 0 && r < bw && c < r) ? __ldcg(A + (k0 + r) * ld + k0 + c) * __ldcg(dv + c)
                                                   : 0.0;
      }
      if (tid < 32) sm.t.b[0][tid] = tid < bw ? __ldcg(dv + tid) : 0.0;
      __syncthreads();
      for (int rr = warp; rr < 32; rr += 4) {
        const int64_t r = 32 * (int64_t)i + rr;
        if (r >= n || bw <= 0) continue;
        double acc = lane < bw ? __ldcg(A + r * ld + k0 + lane) : 0.0;
        for (int c = 0; c < bw; ++c) {
          const double ac = __shfl_sync(0xffffffffu, acc, c);
          if (lane > c) acc = fma(-ac, sm.t.a[lane][c], acc);
        }
        if (lane < bw) A[r * ld + k0 + lane] = acc * sm.t.b[0][lane];
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(solved + i, p + 1);
      }
    } else {
      // tile (i, j) -= L(i rows, panel p) L(j rows, panel p)'
      const int64_t r0 = 32 * (int64_t)i, c0 = 32 * (int64_t)j;
      for (int e = tid; e < 32 * 32; e += kQThreads) {
        const int r = e >> 5, k = e & 31;
        sm.t.a[r][k] = (r0 + r < n && k0 + k < n) ? __ldcg(A + (r0 + r) * ld + k0 + k) : 0.0;
        sm.t.b[r][k] = (c0 + r < n && k0 + k < n) ? __ldcg(A + (c0 + r) * ld + k0 + k) : 0.0;
      }
      __syncthreads();
      // thread: row rr = tid / 4, columns cc = tid % 4 + 4 u
      const int rr = tid >> 2, cq = tid & 3;
      double acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.0;
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        const double a = sm.t.a[rr][k];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fma(a, sm.t.b[cq + 4 * u][k], acc[u]);
      }
      const int64_t r = r0 + rr;
      if (r < n) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t c = c0 + cq + 4 * u;
          if (c < n && (i != j || c <= r)) {
            double* x = A + r * ld + c;
            *x = __ldcg(x) - acc[u];
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(ver + i * nbq + j, p + 1);
      }
    }
  }
}

}  // namespace

cudaError_t launch_chol_queue(const QueueFactor& q, int ctas, cudaStream_t s) {
  if (q.ntasks <= 0) return cudaSuccess;
  if (ctas < 1) ctas = 1;
  chol_queue_kernel<<<(unsigned)ctas, kQThreads, 0, s>>>(q);
  return cudaGetLastError();
}

int chol_queue_ctas() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, chol_queue_kernel, kQThreads, 0) !=
      cudaSuccess)
    return 0;
  return sms * (per > 0 ? per : 1);
}

}  // namespace cpinv

#include "../../include/cpinv.h"

// The queue's failure path without a fault: one task (the diagonal block of
// panel 1 of a 64 x 64 problem) whose input -- tile (1, 1) updated by panel
// 0 -- no task produces, so its bounded wait must run out, record
// ST_TIMEOUT, raise the abort flag and let the launch end.
extern "C" int cpinv_selftest_queue_timeout(void* workspace, size_t workspace_bytes,
                                            void* stream) {
  using namespace cpinv;
  constexpr size_t kNeed = 64 * 1024;
  if (!workspace || workspace_bytes < kNeed || ((uintptr_t)workspace & 255u))
    return CPINV_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = (char*)workspace;
  DevState* st = (DevState*)w;                       // 128 B
  int32_t* head = (int32_t*)(w + 256);               // 2 ints
  int32_t* flags = (int32_t*)(w + 512);              // nb = 2: 4 + 2 + 2 ints
  QueueTask* task = (QueueTask*)(w + 1024);          // 1 task
  double* dinv = (double*)(w + 2048);                // 64 doubles
  uint8_t* acc = (uint8_t*)(w + 3072);               // 64 bytes
  double* A = (double*)(w + 4096);                   // 64 x 64 (never touched)
  DevState h{};
  h.dim_n = 64;
  h.tol = 1.0;
  const QueueTask t{kQDiag, 0, 1, 1, 1, 0};
  if (cudaMemsetAsync(w, 0, kNeed, s) != cudaSuccess ||
      cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(task, &t, sizeof(t), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CPINV_ERR_CUDA;
  QueueFactor q;
  std::memset(&q, 0, sizeof(q));
  q.A = A;
  q.np = 64;
  q.zA = 64 * 64;
  q.sel = SEL_N;
  q.spd = 0;
  q.st = st;
  q.acc = acc;
  q.zAcc = 64;
  q.dinv = dinv;
  q.zDinv = 64;
  q.flags = flags;
  q.zFlags = 8;
  q.nb_max = 2;
  q.ntasks = 1;
  q.tasks = task;
  q.head = head;
  if (launch_chol_queue(q, 2, s) != cudaSuccess) return CPINV_ERR_CUDA;
  DevState r;
  int32_t hd[2];
  if (cudaMemcpyAsync(&r, st, sizeof(r), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hd, head, sizeof(hd), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CPINV_ERR_CUDA;
  return ((r.status & ST_TIMEOUT) && hd[1] == 1) ? CPINV_ERR_TIMEOUT : CPINV_OK;
}
