// Host-side launchers of the cpinv kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cpinv {

// gemm_fp64.cu
cudaError_t launch_dgemm(const GemmParams& p, bool transA, bool transB, cudaStream_t s);

// chol.cu
cudaError_t launch_tol(const double* A, int64_t lda, int64_t n, double rel_tol, DevState* st,
                       cudaStream_t s);
cudaError_t launch_diag_factor(double* A, int64_t lda, Dim nd, int64_t k0, int b, DevState* st,
                               const int64_t* rdev, uint8_t* accepted, double* Z, double* Tinv,
                               int spd, cudaStream_t s);
cudaError_t launch_scan(const uint8_t* accepted, int64_t n, int32_t* colidx, DevState* st,
                        cudaStream_t s);
cudaError_t launch_gather(const double* Lfull, int64_t lda, int64_t n, const int32_t* colidx,
                          double* L, int64_t ldl, cudaStream_t s);
cudaError_t launch_tri_inv_init(double* W, int64_t ldw, int64_t nmax, const int64_t* rdev,
                                const double* Tinv, int b, cudaStream_t s);
cudaError_t launch_mirror(double* C, int64_t ldc, Dim nd, const int64_t* rdev, cudaStream_t s);
cudaError_t launch_copy_mask(const uint8_t* src, uint8_t* dst, int64_t n, cudaStream_t s);

}  // namespace cpinv
