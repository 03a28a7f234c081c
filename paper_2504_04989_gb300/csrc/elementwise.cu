// elementwise.cu -- tensor transpose (Sec. 2) and the masked residual of the
// completion objective ||P_Omega(C - X)||_F^2 (the observation operator of the
// completion problem, Ex. 3), as C-ABI entry points.
#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

// AT(:,:,0) = A(:,:,0)^T, AT(:,:,k) = A(:,:,n3-k)^T for k >= 1; 32 x 32 tiles
// through shared memory so both the reads and the writes are coalesced.
template <typename T>
__global__ void k_ttranspose(const T* __restrict__ A, T* __restrict__ AT, int n1, int n2, int n3) {
  __shared__ T tile[32][33];
  const int k = blockIdx.z;
  const int src = (k == 0) ? 0 : n3 - k;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const T* As = A + (long)src * n1 * n2;
  T* Ad = AT + (long)k * n1 * n2;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    if (i < n1 && j < n2) tile[r][threadIdx.x] = As[(long)i * n2 + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (i < n1 && j < n2) Ad[(long)j * n1 + i] = tile[threadIdx.x][r];
  }
}

// R = M .* (C - X) and per-block partial sums of R^2 (FP64); a second kernel
// adds the partials in a fixed order (deterministic).
constexpr int MR_BLOCKS = 1024;
template <typename T>
__global__ void __launch_bounds__(256) k_masked_residual(const T* __restrict__ C, const T* __restrict__ X,
                                                         const uint8_t* __restrict__ M, T* __restrict__ R, long n,
                                                         double* __restrict__ partial) {
  __shared__ double red[8];
  double acc = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T r = M[i] ? (C[i] - X[i]) : T(0);
    R[i] = r;
    acc += (double)r * (double)r;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double red[8];
  double acc = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace tsvd

using namespace tsvd;

extern "C" int ttranspose(const void* A, void* AT, int n1, int n2, int n3, int precision, void* stream) {
  if (!A || !AT || n1 < 1 || n2 < 1 || n3 < 1) return TSVD_ERR_INVALID_ARG;
  if (precision < TSVD_FP64 || precision > TSVD_MIXED_BF16) return TSVD_ERR_INVALID_ARG;
  if (n3 > 65535) return TSVD_ERR_UNSUPPORTED;
  dim3 grid(cdiv(n2, 32), cdiv(n1, 32), n3), block(32, 8);
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64) k_ttranspose<double><<<grid, block, 0, s>>>((const double*)A, (double*)AT, n1, n2, n3);
  else k_ttranspose<float><<<grid, block, 0, s>>>((const float*)A, (float*)AT, n1, n2, n3);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

extern "C" int tsvd_masked_residual(const void* C, const void* X, const uint8_t* mask, void* R, double* loss,
                                    double* partial, long n, int precision, void* stream) {
  if (!C || !X || !mask || !R || !loss || !partial || n < 0) return TSVD_ERR_INVALID_ARG;
  if (precision < TSVD_FP64 || precision > TSVD_MIXED_BF16) return TSVD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::max<long>(1, std::min<long>(MR_BLOCKS, cdiv(n, 256)));
  if (precision == TSVD_FP64)
    k_masked_residual<double><<<blocks, 256, 0, s>>>((const double*)C, (const double*)X, mask, (double*)R, n, partial);
  else
    k_masked_residual<float><<<blocks, 256, 0, s>>>((const float*)C, (const float*)X, mask, (float*)R, n, partial);
  TSVD_LAUNCHED();
  k_sum_partials<<<1, 256, 0, s>>>(partial, blocks, loss);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
