// cpinv_pinv_static: the pseudoinverse of small matrices with no device
// allocation at all (declared in include/cpinv.h).
//
// Who needs it: callers that cannot call cudaMalloc -- a real-time or
// latency-critical loop in which cudaMalloc / cudaFree would block the host or
// synchronize the device, or a plugin inside a host application that owns all
// GPU memory and hands out no allocator.  Such a caller passes its input and
// output buffers only; the scratch comes from a fixed array compiled into the
// library.
//
// The scratch is one file-scope __device__ array of CPINV_STATIC_SCRATCH_BYTES
// (1 MiB).  Every GPU that loads the library holds it until the process exits.
// Host code may not use the array's name as a device address (on the host it
// is only a stand-in), so the first call on each device looks the real address
// up with cudaGetSymbolAddress, with that device current, and caches it.  The
// cached address is only valid for the context it was looked up in: a device
// reset between calls makes it stale (documented in the header).
//
// Only the FP64 mode fits in the array at every order up to 128; the
// exact-slice mode's tensor-core residue buffers exceed it at any size, so
// those calls (and BF16x3 calls above order ~32) are refused by the size
// check before any GPU work.
#include <cstdint>
#include <mutex>
#include <unordered_map>

#include "../../include/cpinv.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = CPINV_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_setup_mu;
std::unordered_map<int, void*> g_scratch_addr;  // device ordinal -> device address

// Set-up, once per device (the current one): the device address of the array.
int scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CPINV_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  auto it = g_scratch_addr.find(dev);
  if (it != g_scratch_addr.end()) {
    *out = it->second;
    return CPINV_OK;
  }
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr)
    return CPINV_ERR_CUDA;
  g_scratch_addr.emplace(dev, ptr);
  *out = ptr;
  return CPINV_OK;
}

}  // namespace

extern "C" int cpinv_pinv_static(const double* G, int64_t m, int64_t n, int64_t ldg, double* Gp,
                                 int64_t ldgp, const cpinv_opts* o, int64_t* rank_out,
                                 void* stream) {
  if (rank_out) *rank_out = -1;
  if (m < 0 || n < 0) return CPINV_ERR_INVALID_ARG;
  const int64_t order = m < n ? m : n;
  if (order > CPINV_STATIC_MAX_ORDER) return CPINV_ERR_UNSUPPORTED;
  const size_t need = cpinv_pinv_workspace_size(m, n, o);
  if (need == 0) return CPINV_ERR_INVALID_ARG;
  if (need > kScratchBytes) return CPINV_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  if (m > 0 && n > 0) {
    const int rc = scratch_for_current_device(&scratch);
    if (rc != CPINV_OK) return rc;
  }
  // The pipeline clears the per-call state it reads before writing it (the
  // rank, status and tolerance record is zeroed on the stream first), so the
  // previous call's contents of the array do no harm.  Kernels are launched
  // directly: no CUDA graph is instantiated on this path.
  cpinv::NoGraphScope direct_launches;
  return cpinv_pinv(G, m, n, ldg, Gp, ldgp, scratch, kScratchBytes, o, rank_out, stream);
}
