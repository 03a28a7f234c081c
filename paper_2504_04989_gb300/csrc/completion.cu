// completion.cu -- the pieces of the data-completion iteration of Ex. 3
// (Sec. 5) that run between two T-SVDs, as C-ABI entry points:
//   X^(n)   = U * S * V^T       (the low-rank approximation L(C^(n)) from the
//                                factors of Alg. 2: per Fourier slice
//                                X_k = U_k diag(S_k) V_k^H, then the inverse
//                                transform; Alg. TP for the products)
//   C^(n+1) = T .* M + (1 - T) .* X^(n)   (T the observation mask, M the data)
// and the tubes of S^p (p = 1 or 1/2) from the Fourier-domain singular values,
// and the squared distance of two tensors (for the PSNR of Sec. 5).
#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

// Uh (h x n1 x R per slice) columns scaled by the complex tube values Sh (h x R)
template <typename C>
__global__ void k_scale_by_tubes(C* __restrict__ Uh, const C* __restrict__ Sh, int n1, int R, int h) {
  const long total = (long)h * n1 * R;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int r = idx % R;
    const long k = idx / ((long)n1 * R);
    Uh[idx] = cmul(Uh[idx], Sh[k * R + r]);
  }
}

// tubes of S^p: Sh[k][r] = sigma_hat[k][r]^p (real), for the inverse transform
template <typename C>
__global__ void k_sigma_power(const double* __restrict__ sig, long n, double p, C* __restrict__ Sh) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = fmax(sig[i], 0.0);
  const double v = (p == 1.0) ? s : (p == 0.5) ? sqrt(s) : pow(s, p);
  Sh[i] = from_c64<C>(make_double2(v, 0.0));
}

// C <- T ? M : X and per-block partial sums of (C_new - C_old)^2 in FP64
template <typename T>
__global__ void __launch_bounds__(256) k_fill_in(T* __restrict__ Cm, const T* __restrict__ M,
                                                 const uint8_t* __restrict__ mask, const T* __restrict__ X, long n,
                                                 double* __restrict__ partial) {
  __shared__ double red[8];
  double acc = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T c = mask[i] ? M[i] : X[i];
    const double d = (double)c - (double)Cm[i];
    acc += d * d;
    Cm[i] = c;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// per-block partial sums of (A - B)^2 in FP64
template <typename T>
__global__ void __launch_bounds__(256) k_sqdiff(const T* __restrict__ A, const T* __restrict__ B, long n,
                                                double* __restrict__ partial) {
  __shared__ double red[8];
  double acc = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double d = (double)A[i] - (double)B[i];
    acc += d * d;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_partials_to(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double red[8];
  double acc = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];  // fixed order per thread
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) *out = s;
}

constexpr int RED_BLOCKS = 1024;  // partial-sum slots the reductions use (the caller's `partial` array)

template <typename T>
struct LrWs {
  cx_t<T>*Uh, *Vh, *Sh, *Xh;
  void* sk;
  size_t sk_elems;
  size_t bytes;
};

template <typename T>
static LrWs<T> carve_lr(void* base, int n1, int n2, int n3, int R) {
  using C = cx_t<T>;
  const size_t h = n3 / 2 + 1;
  Carver cv(base);
  LrWs<T> w;
  w.Uh = cv.take<C>(h * n1 * R);
  w.Vh = cv.take<C>(h * n2 * R);
  w.Sh = cv.take<C>(h * R);
  w.Xh = cv.take<C>(h * n1 * n2);
  w.sk_elems = std::min<size_t>((size_t)1 << 20, 4 * h * (size_t)n1 * n2);
  w.sk = cv.take<C>(w.sk_elems);
  w.bytes = cv.bytes();
  return w;
}

template <typename T>
static int lowrank_run(const T* U, const T* S, const T* V, int n1, int n2, int n3, int R, T* X, void* ws,
                       cudaStream_t s) {
  using C = cx_t<T>;
  LrWs<T> w = carve_lr<T>(ws, n1, n2, n3, R);
  const int h = n3 / 2 + 1;
  TSVD_TRY(launch_rfft3<T>(U, w.Uh, (long)n1 * R, n3, s));
  TSVD_TRY(launch_rfft3<T>(V, w.Vh, (long)n2 * R, n3, s));
  TSVD_TRY(launch_rfft3<T>(S, w.Sh, (long)R, n3, s));
  const long total = (long)h * n1 * R;
  k_scale_by_tubes<C><<<std::min<long>(cdiv(total, 256), 4096), 256, 0, s>>>(w.Uh, w.Sh, n1, R, h);
  TSVD_LAUNCHED();
  TSVD_TRY(cgemm<C>(gemm('N', 'H', n1, n2, R, 1.0, w.Uh, R, (long)n1 * R, w.Vh, R, (long)n2 * R, 0.0, w.Xh, n2,
                         (long)n1 * n2, h),
                    w.sk, w.sk_elems, s));
  return launch_irfft3<T>(w.Xh, X, (long)n1 * n2, n3, s);
}

}  // namespace tsvd

using namespace tsvd;

extern "C" int tsvd_lowrank_workspace_size(int n1, int n2, int n3, int R, int precision, size_t* bytes) {
  if (!bytes || n1 < 1 || n2 < 1 || n3 < 1 || R < 1) return TSVD_ERR_INVALID_ARG;
  if (precision == TSVD_FP64) *bytes = carve_lr<double>(nullptr, n1, n2, n3, R).bytes;
  else if (precision == TSVD_FP32) *bytes = carve_lr<float>(nullptr, n1, n2, n3, R).bytes;
  else return TSVD_ERR_INVALID_ARG;
  return TSVD_OK;
}

extern "C" int tsvd_lowrank(const void* U, const void* S, const void* V, int n1, int n2, int n3, int R, int precision,
                            void* X, void* ws, size_t ws_bytes, void* stream) {
  size_t need = 0;
  TSVD_TRY(tsvd_lowrank_workspace_size(n1, n2, n3, R, precision, &need));
  if (!U || !S || !V || !X || !ws || ((uintptr_t)ws & 255) != 0) return TSVD_ERR_INVALID_ARG;
  if (ws_bytes < need) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64)
    return lowrank_run<double>((const double*)U, (const double*)S, (const double*)V, n1, n2, n3, R, (double*)X, ws,
                               s);
  return lowrank_run<float>((const float*)U, (const float*)S, (const float*)V, n1, n2, n3, R, (float*)X, ws, s);
}

extern "C" int tsvd_sigma_tubes(const double* sigma_hat, int R, int n3, double power, int precision, void* tubes,
                                void* ws, size_t ws_bytes, void* stream) {
  if (!sigma_hat || !tubes || !ws || R < 1 || n3 < 1 || !(power > 0.0)) return TSVD_ERR_INVALID_ARG;
  if (precision != TSVD_FP64 && precision != TSVD_FP32) return TSVD_ERR_INVALID_ARG;
  const long n = (long)(n3 / 2 + 1) * R;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64) {
    if (ws_bytes < (size_t)n * sizeof(double2)) return TSVD_ERR_WORKSPACE;
    k_sigma_power<double2><<<cdiv(n, 256), 256, 0, s>>>(sigma_hat, n, power, (double2*)ws);
    TSVD_LAUNCHED();
    return launch_irfft3<double>((const double2*)ws, (double*)tubes, R, n3, s);
  }
  if (ws_bytes < (size_t)n * sizeof(float2)) return TSVD_ERR_WORKSPACE;
  k_sigma_power<float2><<<cdiv(n, 256), 256, 0, s>>>(sigma_hat, n, power, (float2*)ws);
  TSVD_LAUNCHED();
  return launch_irfft3<float>((const float2*)ws, (float*)tubes, R, n3, s);
}

extern "C" int tsvd_fill_in(void* Cm, const void* M, const uint8_t* mask, const void* X, long n, int precision,
                            double* partial, double* change2, void* stream) {
  if (!Cm || !M || !mask || !X || !partial || !change2 || n < 0) return TSVD_ERR_INVALID_ARG;
  if (precision != TSVD_FP64 && precision != TSVD_FP32) return TSVD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::max<long>(1, std::min<long>(RED_BLOCKS, cdiv(n, 256)));
  if (precision == TSVD_FP64)
    k_fill_in<double><<<blocks, 256, 0, s>>>((double*)Cm, (const double*)M, mask, (const double*)X, n, partial);
  else
    k_fill_in<float><<<blocks, 256, 0, s>>>((float*)Cm, (const float*)M, mask, (const float*)X, n, partial);
  TSVD_LAUNCHED();
  k_sum_partials_to<<<1, 256, 0, s>>>(partial, blocks, change2);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

extern "C" int tsvd_sqdiff(const void* A, const void* B, long n, int precision, double* partial, double* out,
                           void* stream) {
  if (!A || !B || !partial || !out || n < 0) return TSVD_ERR_INVALID_ARG;
  if (precision != TSVD_FP64 && precision != TSVD_FP32) return TSVD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::max<long>(1, std::min<long>(RED_BLOCKS, cdiv(n, 256)));
  if (precision == TSVD_FP64)
    k_sqdiff<double><<<blocks, 256, 0, s>>>((const double*)A, (const double*)B, n, partial);
  else
    k_sqdiff<float><<<blocks, 256, 0, s>>>((const float*)A, (const float*)B, n, partial);
  TSVD_LAUNCHED();
  k_sum_partials_to<<<1, 256, 0, s>>>(partial, blocks, out);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
