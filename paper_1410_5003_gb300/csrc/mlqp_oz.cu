// Test hook of the FP64 tensor-core products (mlqp_oz.cuh) on plain
// column-major operands: C -= A B for a rows x K block A, a K x cols block B;
// K <= 16 by the block LU's update kernel, 16 < K <= 128 by the chunked one.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mlqp.h"
#include "mlqp_oz.cuh"

namespace mlqp {

struct OzPlain {
  const double2* A;
  const double2* B;
  double2* C;
  int lda, ldb, ldc, rows, cols, K, v0_, u0_;
  __device__ bool setup() {
    const int tc = (cols + OZ_TILE - 1) / OZ_TILE;
    v0_ = (blockIdx.x / tc) * OZ_TILE;
    u0_ = (blockIdx.x % tc) * OZ_TILE;
    return v0_ < rows;
  }
  __device__ int v0() const { return v0_; }
  __device__ int u0() const { return u0_; }
  __device__ int nk() const { return K; }
  __device__ double2 a(int v, int k) const {
    return (v < rows && k < K) ? A[(size_t)k * lda + v] : make_double2(0.0, 0.0);
  }
  __device__ double2 b(int k, int u) const {
    return (u < cols && k < K) ? B[(size_t)u * ldb + k] : make_double2(0.0, 0.0);
  }
  __device__ OzRow row(int v) const { return OzRow{C + v, 0, v < rows ? cols : 0, true}; }
  __device__ long long col_off(bool, int u) const { return (long long)u * ldc; }
};

}  // namespace mlqp

extern "C" mlqp_status mlqp_debug_oz_update(const void* d_A, int lda, const void* d_B, int ldb, void* d_C, int ldc,
                                            int rows, int cols, int K, void* d_work, void* stream) {
  using namespace mlqp;
  if (!d_A || !d_B || !d_C || !d_work || rows < 1 || cols < 1 || K < 1 || K > 128 || lda < rows || ldb < K ||
      ldc < rows)
    return MLQP_EINVAL;
  if (((uintptr_t)d_A | (uintptr_t)d_B | (uintptr_t)d_C | (uintptr_t)d_work) & 15u) return MLQP_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(d_work);
  cudaError_t e = cudaFuncSetAttribute(k_oz_update<OzPlain>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)OZ_SMEM_LAUNCH);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_oz_gemm<OzPlain>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM_LAUNCH);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return MLQP_ECUDA;
  OzPlain g{static_cast<const double2*>(d_A), static_cast<const double2*>(d_B), static_cast<double2*>(d_C),
            lda, ldb, ldc, rows, cols, K, 0, 0};
  const int tiles = ((rows + OZ_TILE - 1) / OZ_TILE) * ((cols + OZ_TILE - 1) / OZ_TILE);
  if (K <= 16)
    k_oz_update<OzPlain><<<tiles, OZ_THREADS, OZ_SMEM_LAUNCH, st>>>(g, status);
  else  // longer inner dimensions in chunks of 16 (the Schur updates' kernel)
    k_oz_gemm<OzPlain><<<tiles, OZ_THREADS, OZ_SMEM_LAUNCH, st>>>(g, status);
  int hs = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return MLQP_ECUDA;
  return hs ? static_cast<mlqp_status>(hs) : MLQP_OK;
}
