// tqr.cu -- T-QR (Alg. TQR) and the Moore-Penrose pseudoinverse (Alg. mp) of
// Sec. 2 on the per-slice kernels of the T-SVD, as C-ABI entry points.
//
// Both work on the h = floor(n3/2)+1 non-redundant Fourier slices (the others
// are their conjugates, restored by the inverse transform):
//   T-QR:  X_k = Q_k R_k, economy size p = min(n1, n2): the first p columns of
//          X_k are orthonormalised block by block (128 columns at a time) by
//          the block step of the Krylov basis (classical Gram-Schmidt against
//          the finished columns + shifted CholeskyQR3, dependent columns
//          replaced), then R_k = Q_k^H X_k with its strict lower part set to
//          zero and its diagonal to its real part (CholeskyQR's triangular
//          factors have a positive real diagonal, so diag(R) >= 0).
//   pinv:  M_k = X_k (n1 >= n2) or X_k^H (n1 < n2), M_k = Q_k R_k as above,
//          R_k^{-1} by inverting its 32 x 32 diagonal blocks and a block back
//          substitution, then X_k^+ = R_k^{-1} Q_k^H (tall) or Q_k R_k^{-H}
//          (wide, pinv(X) = pinv(X^H)^H).  This is the pseudoinverse when
//          every slice has full rank min(n1, n2); rank-deficient slices are
//          detected at the CholeskyQR pivots and reported.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

constexpr int TQR_B = 128;                       // column block of the orthonormalisation
constexpr int TRI_B = 32;                        // diagonal block of the triangular inverse (one warp)
constexpr uint64_t TQR_REPAIR_SEED = 0x7151ull;  // Philox key of replacement directions

// batched conjugate transpose: dst_b (cols x rows) = src_b (rows x cols)^H
template <typename C>
__global__ void __launch_bounds__(256) k_conj_transpose(const C* __restrict__ src, C* __restrict__ dst, int rows,
                                                        int cols) {
  __shared__ C tile[32][33];
  const long b = blockIdx.z;
  src += b * (long)rows * cols;
  dst += b * (long)rows * cols;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = src[(long)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[(long)c * rows + r] = cconj(tile[threadIdx.x][i]);
  }
}

// R (rows x cols per slice): zero below the diagonal, real diagonal
template <typename T>
__global__ void k_triu_realdiag(cx_t<T>* __restrict__ R, int rows, int cols, int batch) {
  const long total = (long)batch * rows * cols;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = idx % cols;
    const int i = (idx / cols) % rows;
    if (i > j) R[idx] = mkc(T(0), T(0));
    else if (i == j) R[idx].y = T(0);
  }
}

// Inverses of the diagonal blocks (TRI_B x TRI_B, the last one ragged) of the
// upper triangular R (p x p per slice), written into the same blocks of Rinv:
// thread j solves R_II x = e_j by back substitution (x_i = 0 for i > j).
template <typename C>
__global__ void __launch_bounds__(TRI_B) k_trtri_diag(const C* __restrict__ R, C* __restrict__ Rinv, int p) {
  using Rt = decltype(C().x);
  __shared__ C Rs[TRI_B][TRI_B + 1];
  __shared__ C Xs[TRI_B][TRI_B + 1];  // Xs[i][j]: row i of column j of the inverse
  const int I = blockIdx.x;
  const long b = blockIdx.y;
  const int r0 = I * TRI_B, nb = min(TRI_B, p - r0);
  R += b * (long)p * p;
  Rinv += b * (long)p * p;
  const int j = threadIdx.x;
  for (int i = 0; i < nb; ++i)
    if (j < nb) Rs[i][j] = R[(long)(r0 + i) * p + r0 + j];
  __syncthreads();
  if (j < nb) {
    for (int i = nb - 1; i >= 0; --i) {
      C acc = mkc(Rt(i == j ? 1 : 0), Rt(0));
      if (i > j) {
        Xs[i][j] = mkc(Rt(0), Rt(0));
        continue;
      }
      for (int k = i + 1; k <= j; ++k) acc = csub(acc, cmul(Rs[i][k], Xs[k][j]));
      // x_i = acc / R_ii
      const C d = Rs[i][i];
      const Rt den = d.x * d.x + d.y * d.y;
      Xs[i][j] = (den > Rt(0)) ? mkc((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den)
                               : mkc(Rt(0), Rt(0));
    }
  }
  __syncthreads();
  for (int i = 0; i < nb; ++i)
    if (j < nb) Rinv[(long)(r0 + i) * p + r0 + j] = Xs[i][j];
}

template <typename T>
struct TqrWs {
  using C = cx_t<T>;
  C* Ah;     // h x n1 x n2 half spectrum of X
  C* Mt;     // h x n2 x n1: X_k^H (pinv of a wide X), else unused
  C* Q;      // h x Mr x p
  C* W;      // h x Mr x b
  C* P;      // h x p x b
  C* G;      // h x b x b
  C* Minv;   // h x b x b
  C* Rh;     // h x p x Nc
  C* Rinv;   // h x p x p (pinv)
  C* Tm;     // h x TRI_B x p (pinv)
  C* Xp;     // h x n2 x n1 (pinv)
  uint32_t* dead;
  int* counters;
  double2* splitk;
  size_t splitk_elems;  // double2 elements
  size_t bytes;
};

struct TqrDims {
  int n1, n2, n3, h, Mr, Nc, p, b;
  bool wide;  // pinv of a wide X: M = X^H
};

static int tqr_dims(int n1, int n2, int n3, int precision, bool pinv, TqrDims* d) {
  if (n1 < 1 || n2 < 1 || n3 < 1) return TSVD_ERR_INVALID_ARG;
  if (precision != TSVD_FP64 && precision != TSVD_FP32) return TSVD_ERR_INVALID_ARG;
  d->n1 = n1;
  d->n2 = n2;
  d->n3 = n3;
  d->h = n3 / 2 + 1;
  d->wide = pinv && n1 < n2;
  d->Mr = d->wide ? n2 : n1;
  d->Nc = d->wide ? n1 : n2;
  d->p = std::min(n1, n2);
  d->b = std::min(TQR_B, d->p);
  if ((double)d->h * n1 * n2 > (double)(1L << 36) || (double)d->h * d->p * d->p > (double)(1L << 36))
    return TSVD_ERR_UNSUPPORTED;
  if (d->h > 65535) return TSVD_ERR_UNSUPPORTED;
  return TSVD_OK;
}

template <typename T>
static TqrWs<T> carve_tqr(void* base, const TqrDims& d, bool pinv) {
  using C = cx_t<T>;
  Carver cv(base);
  TqrWs<T> w;
  const size_t h = d.h;
  w.Ah = cv.take<C>(h * d.n1 * d.n2);
  w.Mt = d.wide ? cv.take<C>(h * d.n1 * d.n2) : nullptr;
  w.Q = cv.take<C>(h * d.Mr * d.p);
  w.W = cv.take<C>(h * d.Mr * d.b);
  w.P = cv.take<C>(h * d.p * d.b);
  w.G = cv.take<C>(h * d.b * d.b);
  w.Minv = cv.take<C>(h * d.b * d.b);
  w.Rh = cv.take<C>(h * d.p * d.Nc);
  w.Rinv = pinv ? cv.take<C>(h * d.p * d.p) : nullptr;
  w.Tm = pinv ? cv.take<C>(h * TRI_B * d.p) : nullptr;
  w.Xp = pinv ? cv.take<C>(h * d.n2 * d.n1) : nullptr;
  w.dead = cv.take<uint32_t>(h * 4);
  w.counters = cv.take<int>(8);
  w.splitk_elems = std::min<size_t>((size_t)1 << 22, 8 * h * (size_t)d.p * std::max(d.b, 64));
  w.splitk = cv.take<double2>(w.splitk_elems);
  w.bytes = cv.bytes();
  return w;
}

// Q (Mr x p) and R (p x Nc) of the per-slice matrices M (Mr x Nc, leading dim Nc)
template <typename T>
static int tqr_factor(const TqrDims& d, TqrWs<T>& w, const cx_t<T>* M, cudaStream_t s) {
  using C = cx_t<T>;
  const int Mr = d.Mr, Nc = d.Nc, p = d.p, b = d.b, h = d.h;
  const size_t sk = std::is_same<T, double>::value ? w.splitk_elems : 2 * w.splitk_elems;
  if (cudaMemsetAsync(w.counters, 0, 8 * sizeof(int), s) != cudaSuccess) return TSVD_ERR_CUDA;
  OrthWs o;
  o.Q = w.Q;
  o.W = w.W;
  o.P = w.P;
  o.G = w.G;
  o.Minv = w.Minv;
  o.dead = w.dead;
  o.dead_count = w.counters + 1;
  o.Qt = nullptr;
  o.splitk = w.splitk;
  o.splitk_elems = w.splitk_elems;
  o.k0 = 0;
  o.nyq = (d.n3 % 2 == 0) ? d.n3 / 2 : -1;
  o.tc = nullptr;
  for (int c = 0; c < p; c += b) {
    const int nb = std::min(b, p - c);
    TSVD_TRY(copy_cx<C>(M + c, Nc, (long)Mr * Nc, w.W, b, (long)Mr * b, Mr, nb, h, s));
    TSVD_TRY(orth_block_cols<T>(Mr, b, p, h, o, c, nb, c / b, TQR_REPAIR_SEED, s));
  }
  // R = Q^H M, upper trapezoidal with a real diagonal
  TSVD_TRY(cgemm<C>(gemm('H', 'N', p, Nc, Mr, 1.0, w.Q, p, (long)Mr * p, M, Nc, (long)Mr * Nc, 0.0, w.Rh, Nc,
                         (long)p * Nc, h),
                    w.splitk, sk, s));
  const long total = (long)h * p * Nc;
  k_triu_realdiag<T><<<std::min<long>(cdiv(total, 256), 8192), 256, 0, s>>>(w.Rh, p, Nc, h);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// status of the call into *info (synchronises): dead columns found at the
// CholeskyQR pivots; for the pseudoinverse they mean a rank-deficient slice
static int read_status(int* counters, cudaStream_t s, tsvd_info* info, int p, bool need_full_rank) {
  if (!info) return TSVD_OK;
  int host[8];
  if (cudaMemcpyAsync(host, counters, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TSVD_ERR_CUDA;
  info->status = (need_full_rank && host[1] > 0) ? TSVD_ERR_RANK_DEFICIENT : TSVD_OK;
  info->dead_columns = host[1];
  info->m_eff = p;
  info->reserved = 0;
  return TSVD_OK;
}

template <typename T>
static int tqr_run(const T* A, const TqrDims& d, T* Qout, T* Rout, void* ws, cudaStream_t s, tsvd_info* info) {
  TqrWs<T> w = carve_tqr<T>(ws, d, false);
  TSVD_TRY(launch_rfft3<T>(A, w.Ah, (long)d.n1 * d.n2, d.n3, s));
  TSVD_TRY(tqr_factor<T>(d, w, w.Ah, s));
  TSVD_TRY(launch_irfft3<T>(w.Q, Qout, (long)d.n1 * d.p, d.n3, s));
  TSVD_TRY(launch_irfft3<T>(w.Rh, Rout, (long)d.p * d.n2, d.n3, s));
  return read_status(w.counters, s, info, d.p, false);
}

template <typename T>
static int tpinv_run(const T* A, const TqrDims& d, T* Xout, void* ws, cudaStream_t s, tsvd_info* info) {
  using C = cx_t<T>;
  TqrWs<T> w = carve_tqr<T>(ws, d, true);
  const int p = d.p, Mr = d.Mr, h = d.h;
  const long sP = (long)p * p;
  const size_t sk = std::is_same<T, double>::value ? w.splitk_elems : 2 * w.splitk_elems;
  TSVD_TRY(launch_rfft3<T>(A, w.Ah, (long)d.n1 * d.n2, d.n3, s));
  const C* M = w.Ah;
  if (d.wide) {
    k_conj_transpose<C><<<dim3(cdiv(d.n2, 32), cdiv(d.n1, 32), h), dim3(32, 8), 0, s>>>(w.Ah, w.Mt, d.n1, d.n2);
    TSVD_LAUNCHED();
    M = w.Mt;
  }
  TSVD_TRY(tqr_factor<T>(d, w, M, s));  // R is p x p (Nc = p)
  // R^{-1}: diagonal blocks, then block rows bottom-up:
  //   Rinv(I, e:p) = -Rinv_II (R(I, e:p) Rinv(e:p, e:p)),  e = end of block I
  if (cudaMemsetAsync(w.Rinv, 0, sizeof(C) * (size_t)h * sP, s) != cudaSuccess) return TSVD_ERR_CUDA;
  const int nblk = (int)cdiv(p, TRI_B);
  k_trtri_diag<C><<<dim3(nblk, h), TRI_B, 0, s>>>(w.Rh, w.Rinv, p);
  TSVD_LAUNCHED();
  for (int I = nblk - 2; I >= 0; --I) {
    const int r0 = I * TRI_B, e = r0 + TRI_B, rest = p - e;
    TSVD_TRY(cgemm<C>(gemm('N', 'N', TRI_B, rest, rest, 1.0, w.Rh + (long)r0 * p + e, p, sP, w.Rinv + (long)e * p + e,
                           p, sP, 0.0, w.Tm, p, (long)TRI_B * p, h),
                      w.splitk, sk, s));
    TSVD_TRY(cgemm<C>(gemm('N', 'N', TRI_B, rest, TRI_B, -1.0, w.Rinv + (long)r0 * p + r0, p, sP, w.Tm, p,
                           (long)TRI_B * p, 0.0, w.Rinv + (long)r0 * p + e, p, sP, h),
                      w.splitk, sk, s));
  }
  // X^+ = R^{-1} Q^H (p x Mr = n2 x n1) or Q R^{-H} (Mr x p = n2 x n1)
  const long sX = (long)d.n2 * d.n1;
  if (!d.wide)
    TSVD_TRY(cgemm<C>(gemm('N', 'H', p, Mr, p, 1.0, w.Rinv, p, sP, w.Q, p, (long)Mr * p, 0.0, w.Xp, d.n1, sX, h),
                      w.splitk, sk, s));
  else
    TSVD_TRY(cgemm<C>(gemm('N', 'H', Mr, p, p, 1.0, w.Q, p, (long)Mr * p, w.Rinv, p, sP, 0.0, w.Xp, d.n1, sX, h),
                      w.splitk, sk, s));
  TSVD_TRY(launch_irfft3<T>(w.Xp, Xout, sX, d.n3, s));
  return read_status(w.counters, s, info, p, true);
}

}  // namespace tsvd

using namespace tsvd;

extern "C" int tqr_workspace_size(int n1, int n2, int n3, int precision, size_t* bytes) {
  if (!bytes) return TSVD_ERR_INVALID_ARG;
  TqrDims d;
  TSVD_TRY(tqr_dims(n1, n2, n3, precision, false, &d));
  *bytes = precision == TSVD_FP64 ? carve_tqr<double>(nullptr, d, false).bytes : carve_tqr<float>(nullptr, d, false).bytes;
  return TSVD_OK;
}

extern "C" int tqr(const void* A, int n1, int n2, int n3, int precision, void* Q, void* R, void* ws, size_t ws_bytes,
                   void* stream, tsvd_info* info) {
  TqrDims d;
  TSVD_TRY(tqr_dims(n1, n2, n3, precision, false, &d));
  if (!A || !Q || !R || !ws || ((uintptr_t)ws & 255) != 0) return TSVD_ERR_INVALID_ARG;
  size_t need = 0;
  TSVD_TRY(tqr_workspace_size(n1, n2, n3, precision, &need));
  if (ws_bytes < need) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64) return tqr_run<double>((const double*)A, d, (double*)Q, (double*)R, ws, s, info);
  return tqr_run<float>((const float*)A, d, (float*)Q, (float*)R, ws, s, info);
}

extern "C" int tpinv_workspace_size(int n1, int n2, int n3, int precision, size_t* bytes) {
  if (!bytes) return TSVD_ERR_INVALID_ARG;
  TqrDims d;
  TSVD_TRY(tqr_dims(n1, n2, n3, precision, true, &d));
  *bytes = precision == TSVD_FP64 ? carve_tqr<double>(nullptr, d, true).bytes : carve_tqr<float>(nullptr, d, true).bytes;
  return TSVD_OK;
}

extern "C" int tpinv(const void* A, int n1, int n2, int n3, int precision, void* X, void* ws, size_t ws_bytes,
                     void* stream, tsvd_info* info) {
  TqrDims d;
  TSVD_TRY(tqr_dims(n1, n2, n3, precision, true, &d));
  if (!A || !X || !ws || ((uintptr_t)ws & 255) != 0) return TSVD_ERR_INVALID_ARG;
  size_t need = 0;
  TSVD_TRY(tpinv_workspace_size(n1, n2, n3, precision, &need));
  if (ws_bytes < need) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64) return tpinv_run<double>((const double*)A, d, (double*)X, ws, s, info);
  return tpinv_run<float>((const float*)A, d, (float*)X, ws, s, info);
}
