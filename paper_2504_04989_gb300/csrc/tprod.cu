// tprod.cu -- t-product (Definition of the T-product and Alg. TP, Sec. 2) and
// its adjoints, as C-ABI entry points.
//
// Forward:  C_k = A_k B_k on the h = floor(n3/2)+1 non-redundant Fourier
//           slices, then the conjugate mirror + inverse transform (Alg. TP).
// Backward: for L = <dC, A*B>, bcirc(X^T) = bcirc(X)^T (Lemma on bcirc) makes
//           the adjoint the t-product with the transpose, whose Fourier slice
//           is the conjugate transpose:  dA_k = dC_k B_k^H,  dB_k = A_k^H dC_k.
// Projection Y = Q*Q^T*A (Sec. 4, the lemma equating the Alg. 2 residual with A - Q (Q^T A)_k): dA_k = Q_k (Q_k^H dY_k),
//           dQ_k = dY_k (A_k^H Q_k) + A_k (dY_k^H Q_k).
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

static int check_prec(int precision) {
  if (precision == TSVD_FP64 || precision == TSVD_FP32) return TSVD_OK;
  if (precision >= TSVD_MIXED_TF32 && precision <= TSVD_SPLIT_TF32) return TSVD_ERR_UNSUPPORTED;
  return TSVD_ERR_INVALID_ARG;
}

static int check_prec_fwd(int precision) {
  if (precision >= TSVD_FP64 && precision <= TSVD_SPLIT_TF32) return TSVD_OK;
  return TSVD_ERR_INVALID_ARG;
}

static GemmArgs gm(char opA, char opB, int M, int N, int K, double alpha, const void* A, long lda, const void* B,
                   long ldb, double beta, void* Cm, long ldc, int batch) {
  GemmArgs g;
  g.opA = opA;
  g.opB = opB;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = alpha;
  g.beta = beta;
  g.A = A;
  g.lda = lda;
  g.sA = (long)(opA == 'N' ? M : K) * lda;
  g.B = B;
  g.ldb = ldb;
  g.sB = (long)(opB == 'N' ? K : N) * ldb;
  g.C = Cm;
  g.ldc = ldc;
  g.sC = (long)M * ldc;
  g.batch = batch;
  return g;
}

constexpr size_t SPLITK_ELEMS = (size_t)1 << 22;  // complex elements of split-K scratch

// ---------------------------------------------------------------------------
template <typename T>
struct TprodWs {
  cx_t<T>*Ah, *Bh, *Ch;
  void* sk;
  size_t bytes;
};
template <typename T>
static TprodWs<T> carve_tprod(void* base, int n1, int n2, int n4, int n3) {
  Carver cv(base);
  const size_t h = n3 / 2 + 1;
  TprodWs<T> w;
  w.Ah = cv.take<cx_t<T>>(h * n1 * n2);
  w.Bh = cv.take<cx_t<T>>(h * n2 * n4);
  w.Ch = cv.take<cx_t<T>>(h * n1 * n4);
  w.sk = cv.take<cx_t<T>>(SPLITK_ELEMS);
  w.bytes = cv.bytes();
  return w;
}

template <typename T>
static int tprod_run(const T* A, const T* B, T* Cout, int n1, int n2, int n4, int n3, void* ws, cudaStream_t s) {
  TprodWs<T> w = carve_tprod<T>(ws, n1, n2, n4, n3);
  const int h = n3 / 2 + 1;
  {
    TSVD_STAGE("tprod_rfft", s);
    TSVD_TRY(launch_rfft3<T>(A, w.Ah, (long)n1 * n2, n3, s));
    TSVD_TRY(launch_rfft3<T>(B, w.Bh, (long)n2 * n4, n3, s));
  }
  {
    TSVD_STAGE("tprod_gemm", s);
    TSVD_TRY(cgemm<cx_t<T>>(gm('N', 'N', n1, n4, n2, 1.0, w.Ah, n2, w.Bh, n4, 0.0, w.Ch, n4, h), w.sk, SPLITK_ELEMS,
                            s));
  }
  {
    TSVD_STAGE("tprod_irfft", s);
    TSVD_TRY(launch_irfft3<T>(w.Ch, Cout, (long)n1 * n4, n3, s));
  }
  return TSVD_OK;
}

// Tensor-core forward: the slice products as one real GEMM per slice,
// real(A_k) (n1 x 2n2) times E(B_k)^T, E(B_k) (2n4 x 2n2) the expanded real
// form of B_k; the interleaved complex product comes out directly.
// MODE 0: one TF32 pass, 1: BF16, 2: split TF32 (hi*hi + hi*lo + lo*hi, operands to ~22 bits)
struct TprodTcWs {
  float2 *Ah, *Bh, *Ch;
  void* Aop;  // operand copy (BF16, FP32 with padded rows, or the TF32 hi part) or null
  float* Alo; // split TF32: the lo part of the operand
  void* E;
  float* Elo; // split TF32: the lo part of the expanded B
  int* err;
  long lda, lde;
  size_t bytes;
};
static TprodTcWs carve_tprod_tc(void* base, int n1, int n2, int n4, int n3, int mode) {
  Carver cv(base);
  const size_t h = n3 / 2 + 1;
  TprodTcWs w;
  const long k2 = 2L * n2;
  w.lda = (k2 + 7) / 8 * 8;
  w.lde = w.lda;
  w.Ah = cv.take<float2>(h * n1 * n2);
  w.Bh = cv.take<float2>(h * n2 * n4);
  w.Ch = cv.take<float2>(h * n1 * n4);
  const bool copy = mode != 0 || (k2 % 4 != 0);
  w.Aop = copy ? cv.take<float>(h * n1 * w.lda) : nullptr;  // big enough for either element type
  w.Alo = (mode == 2) ? cv.take<float>(h * n1 * w.lda) : nullptr;
  w.E = cv.take<float>(h * 2 * (size_t)n4 * w.lde);
  w.Elo = (mode == 2) ? cv.take<float>(h * 2 * (size_t)n4 * w.lde) : nullptr;
  w.err = cv.take<int>(4);
  w.bytes = cv.bytes();
  return w;
}

static int tprod_tc_run(const float* A, const float* B, float* Cout, int n1, int n2, int n4, int n3, int mode,
                        void* ws, cudaStream_t s) {
  const bool bf16 = mode == 1;
  TprodTcWs w = carve_tprod_tc(ws, n1, n2, n4, n3, mode);
  const int h = n3 / 2 + 1;
  const long k2 = 2L * n2;
  {
    TSVD_STAGE("tprod_rfft", s);
    TSVD_TRY(launch_rfft3<float>(A, w.Ah, (long)n1 * n2, n3, s));
    TSVD_TRY(launch_rfft3<float>(B, w.Bh, (long)n2 * n4, n3, s));
  }
  {
    TSVD_STAGE("tprod_expand", s);
    if (mode == 2) {  // hi / lo parts of both operands
      TSVD_TRY(expand_thin_split(w.Bh, n4, (long)n2 * n4, n2, n4, (float*)w.E, w.Elo, w.lde, 2L * n4 * w.lde, h, 0,
                                 s));
      TSVD_TRY(split_rows((const float*)w.Ah, k2, (float*)w.Aop, w.Alo, w.lda, (int)k2, (long)h * n1, s));
    } else {
      TSVD_TRY(expand_thin(w.Bh, n4, (long)n2 * n4, n2, n4, w.E, w.lde, 2L * n4 * w.lde, h, 0, bf16, s));
      if (w.Aop)  // BF16 operand, or FP32 rows padded to 16 bytes
        TSVD_TRY(copy_rows((const float*)w.Ah, k2, w.Aop, w.lda, (int)k2, (long)h * n1, bf16, s));
    }
    if (cudaMemsetAsync(w.err, 0, sizeof(int), s) != cudaSuccess) return TSVD_ERR_CUDA;
  }
  {
    TSVD_STAGE("tprod_gemm_tc", s);
    const void* Aop = w.Aop ? w.Aop : (const void*)w.Ah;
    const long lda = w.Aop ? w.lda : k2;
    if (mode == 2)
      TSVD_TRY(tc_gemm_split((const float*)w.Aop, w.Alo, w.lda, (long)n1 * w.lda, n1, (const float*)w.E, w.Elo,
                             w.lde, 2L * n4 * w.lde, 2 * n4, (int)k2, (float*)w.Ch, 2L * n4, 2L * n1 * n4, h, w.err,
                             s));
    else
      TSVD_TRY(tc_gemm(Aop, lda, (long)n1 * lda, n1, w.E, w.lde, 2L * n4 * w.lde, 2 * n4, (int)k2, (float*)w.Ch,
                       2L * n4, 2L * n1 * n4, h, bf16, w.err, s));
  }
  {
    TSVD_STAGE("tprod_irfft", s);
    TSVD_TRY(launch_irfft3<float>(w.Ch, Cout, (long)n1 * n4, n3, s));
  }
  return TSVD_OK;
}

// ---------------------------------------------------------------------------
template <typename T>
struct TbwdWs {
  cx_t<T>*Ah, *Bh, *dCh, *dAh, *dBh;
  void* sk;
  size_t bytes;
};
template <typename T>
static TbwdWs<T> carve_tbwd(void* base, int n1, int n2, int n4, int n3) {
  Carver cv(base);
  const size_t h = n3 / 2 + 1;
  TbwdWs<T> w;
  w.Ah = cv.take<cx_t<T>>(h * n1 * n2);
  w.Bh = cv.take<cx_t<T>>(h * n2 * n4);
  w.dCh = cv.take<cx_t<T>>(h * n1 * n4);
  w.dAh = cv.take<cx_t<T>>(h * n1 * n2);
  w.dBh = cv.take<cx_t<T>>(h * n2 * n4);
  w.sk = cv.take<cx_t<T>>(SPLITK_ELEMS);
  w.bytes = cv.bytes();
  return w;
}

template <typename T>
static int tbwd_run(const T* A, const T* B, const T* dC, T* dA, T* dB, int n1, int n2, int n4, int n3, void* ws,
                    cudaStream_t s) {
  TbwdWs<T> w = carve_tbwd<T>(ws, n1, n2, n4, n3);
  const int h = n3 / 2 + 1;
  TSVD_TRY(launch_rfft3<T>(dC, w.dCh, (long)n1 * n4, n3, s));
  if (dA) {
    TSVD_TRY(launch_rfft3<T>(B, w.Bh, (long)n2 * n4, n3, s));
    TSVD_TRY(cgemm<cx_t<T>>(gm('N', 'H', n1, n2, n4, 1.0, w.dCh, n4, w.Bh, n4, 0.0, w.dAh, n2, h), w.sk, SPLITK_ELEMS,
                            s));
    TSVD_TRY(launch_irfft3<T>(w.dAh, dA, (long)n1 * n2, n3, s));
  }
  if (dB) {
    TSVD_TRY(launch_rfft3<T>(A, w.Ah, (long)n1 * n2, n3, s));
    TSVD_TRY(cgemm<cx_t<T>>(gm('H', 'N', n2, n4, n1, 1.0, w.Ah, n2, w.dCh, n4, 0.0, w.dBh, n4, h), w.sk, SPLITK_ELEMS,
                            s));
    TSVD_TRY(launch_irfft3<T>(w.dBh, dB, (long)n2 * n4, n3, s));
  }
  return TSVD_OK;
}

// ---------------------------------------------------------------------------
template <typename T>
struct TprojWs {
  cx_t<T>*Qh, *Ah, *dYh, *T1, *T2, *dAh, *dQh;
  void* sk;
  size_t bytes;
};
template <typename T>
static TprojWs<T> carve_tproj(void* base, int n1, int m, int n2, int n3) {
  Carver cv(base);
  const size_t h = n3 / 2 + 1;
  TprojWs<T> w;
  w.Qh = cv.take<cx_t<T>>(h * n1 * m);
  w.Ah = cv.take<cx_t<T>>(h * n1 * n2);
  w.dYh = cv.take<cx_t<T>>(h * n1 * n2);
  w.T1 = cv.take<cx_t<T>>(h * (size_t)std::max(m, n2) * std::max(m, n2));
  w.T2 = cv.take<cx_t<T>>(h * (size_t)n2 * m);
  w.dAh = cv.take<cx_t<T>>(h * n1 * n2);
  w.dQh = cv.take<cx_t<T>>(h * n1 * m);
  w.sk = cv.take<cx_t<T>>(SPLITK_ELEMS);
  w.bytes = cv.bytes();
  return w;
}

template <typename T>
static int tproj_run(const T* Q, const T* A, const T* dY, T* dQ, T* dA, int n1, int m, int n2, int n3, void* ws,
                     cudaStream_t s) {
  TprojWs<T> w = carve_tproj<T>(ws, n1, m, n2, n3);
  const int h = n3 / 2 + 1;
  using C = cx_t<T>;
  TSVD_TRY(launch_rfft3<T>(Q, w.Qh, (long)n1 * m, n3, s));
  TSVD_TRY(launch_rfft3<T>(dY, w.dYh, (long)n1 * n2, n3, s));
  if (dA) {
    // T1 = Q^H dY (m x n2); dA = Q T1
    TSVD_TRY(cgemm<C>(gm('H', 'N', m, n2, n1, 1.0, w.Qh, m, w.dYh, n2, 0.0, w.T1, n2, h), w.sk, SPLITK_ELEMS, s));
    TSVD_TRY(cgemm<C>(gm('N', 'N', n1, n2, m, 1.0, w.Qh, m, w.T1, n2, 0.0, w.dAh, n2, h), w.sk, SPLITK_ELEMS, s));
    TSVD_TRY(launch_irfft3<T>(w.dAh, dA, (long)n1 * n2, n3, s));
  }
  if (dQ) {
    TSVD_TRY(launch_rfft3<T>(A, w.Ah, (long)n1 * n2, n3, s));
    // T2 = A^H Q (n2 x m); dQ = dY T2
    TSVD_TRY(cgemm<C>(gm('H', 'N', n2, m, n1, 1.0, w.Ah, n2, w.Qh, m, 0.0, w.T2, m, h), w.sk, SPLITK_ELEMS, s));
    TSVD_TRY(cgemm<C>(gm('N', 'N', n1, m, n2, 1.0, w.dYh, n2, w.T2, m, 0.0, w.dQh, m, h), w.sk, SPLITK_ELEMS, s));
    // T2 = dY^H Q; dQ += A T2
    TSVD_TRY(cgemm<C>(gm('H', 'N', n2, m, n1, 1.0, w.dYh, n2, w.Qh, m, 0.0, w.T2, m, h), w.sk, SPLITK_ELEMS, s));
    TSVD_TRY(cgemm<C>(gm('N', 'N', n1, m, n2, 1.0, w.Ah, n2, w.T2, m, 1.0, w.dQh, m, h), w.sk, SPLITK_ELEMS, s));
    TSVD_TRY(launch_irfft3<T>(w.dQh, dQ, (long)n1 * m, n3, s));
  }
  return TSVD_OK;
}

template <typename T>
static int tproj_fwd_run(const T* Q, const T* A, T* Y, int n1, int m, int n2, int n3, void* ws, cudaStream_t s) {
  TprojWs<T> w = carve_tproj<T>(ws, n1, m, n2, n3);
  const int h = n3 / 2 + 1;
  using C = cx_t<T>;
  TSVD_TRY(launch_rfft3<T>(Q, w.Qh, (long)n1 * m, n3, s));
  TSVD_TRY(launch_rfft3<T>(A, w.Ah, (long)n1 * n2, n3, s));
  TSVD_TRY(cgemm<C>(gm('H', 'N', m, n2, n1, 1.0, w.Qh, m, w.Ah, n2, 0.0, w.T1, n2, h), w.sk, SPLITK_ELEMS, s));
  TSVD_TRY(cgemm<C>(gm('N', 'N', n1, n2, m, 1.0, w.Qh, m, w.T1, n2, 0.0, w.dAh, n2, h), w.sk, SPLITK_ELEMS, s));
  TSVD_TRY(launch_irfft3<T>(w.dAh, Y, (long)n1 * n2, n3, s));
  return TSVD_OK;
}

static bool dims_ok(long a, long b, long c, long d) { return a >= 1 && b >= 1 && c >= 1 && d >= 1; }
static bool aligned(const void* p) { return ((uintptr_t)p & 255) == 0; }

}  // namespace tsvd

using namespace tsvd;

extern "C" int tprod_workspace_size(int n1, int n2, int n4, int n3, int precision, size_t* bytes) {
  if (!bytes || !dims_ok(n1, n2, n4, n3)) return TSVD_ERR_INVALID_ARG;
  TSVD_TRY(check_prec_fwd(precision));
  if (precision == TSVD_FP64) *bytes = carve_tprod<double>(nullptr, n1, n2, n4, n3).bytes;
  else if (precision == TSVD_FP32) *bytes = carve_tprod<float>(nullptr, n1, n2, n4, n3).bytes;
  else *bytes = carve_tprod_tc(nullptr, n1, n2, n4, n3, precision - TSVD_MIXED_TF32).bytes;
  return TSVD_OK;
}

extern "C" int tprod(const void* A, const void* B, void* C, int n1, int n2, int n4, int n3, int precision, void* ws,
                     size_t ws_bytes, void* stream) {
  if (!A || !B || !C || !ws || !dims_ok(n1, n2, n4, n3) || !aligned(ws)) return TSVD_ERR_INVALID_ARG;
  size_t need;
  TSVD_TRY(tprod_workspace_size(n1, n2, n4, n3, precision, &need));
  if (ws_bytes < need) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64)
    return tprod_run<double>((const double*)A, (const double*)B, (double*)C, n1, n2, n4, n3, ws, s);
  if (precision == TSVD_FP32)
    return tprod_run<float>((const float*)A, (const float*)B, (float*)C, n1, n2, n4, n3, ws, s);
  // TF32 (mode 0), BF16 (1), split TF32 (2) on tcgen05
  return tprod_tc_run((const float*)A, (const float*)B, (float*)C, n1, n2, n4, n3, precision - TSVD_MIXED_TF32, ws,
                      s);
}

extern "C" int tprod_backward_workspace_size(int n1, int n2, int n4, int n3, int precision, size_t* bytes) {
  if (!bytes || !dims_ok(n1, n2, n4, n3)) return TSVD_ERR_INVALID_ARG;
  TSVD_TRY(check_prec(precision));
  *bytes = precision == TSVD_FP64 ? carve_tbwd<double>(nullptr, n1, n2, n4, n3).bytes
                                  : carve_tbwd<float>(nullptr, n1, n2, n4, n3).bytes;
  return TSVD_OK;
}

extern "C" int tprod_backward(const void* A, const void* B, const void* dC, void* dA, void* dB, int n1, int n2, int n4,
                              int n3, int precision, void* ws, size_t ws_bytes, void* stream) {
  if (!dC || !ws || !dims_ok(n1, n2, n4, n3) || !aligned(ws)) return TSVD_ERR_INVALID_ARG;
  if ((dA && !B) || (dB && !A)) return TSVD_ERR_INVALID_ARG;
  size_t need;
  TSVD_TRY(tprod_backward_workspace_size(n1, n2, n4, n3, precision, &need));
  if (ws_bytes < need) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64)
    return tbwd_run<double>((const double*)A, (const double*)B, (const double*)dC, (double*)dA, (double*)dB, n1, n2,
                            n4, n3, ws, s);
  return tbwd_run<float>((const float*)A, (const float*)B, (const float*)dC, (float*)dA, (float*)dB, n1, n2, n4, n3,
                         ws, s);
}

extern "C" int tproj_backward_workspace_size(int n1, int m, int n2, int n3, int precision, size_t* bytes) {
  if (!bytes || !dims_ok(n1, m, n2, n3)) return TSVD_ERR_INVALID_ARG;
  TSVD_TRY(check_prec(precision));
  *bytes = precision == TSVD_FP64 ? carve_tproj<double>(nullptr, n1, m, n2, n3).bytes
                                  : carve_tproj<float>(nullptr, n1, m, n2, n3).bytes;
  return TSVD_OK;
}

extern "C" int tproj_backward(const void* Q, const void* A, const void* dY, void* dQ, void* dA, int n1, int m, int n2,
                              int n3, int precision, void* ws, size_t ws_bytes, void* stream) {
  if (!Q || !dY || !ws || !dims_ok(n1, m, n2, n3) || !aligned(ws)) return TSVD_ERR_INVALID_ARG;
  if (dQ && !A) return TSVD_ERR_INVALID_ARG;
  size_t need;
  TSVD_TRY(tproj_backward_workspace_size(n1, m, n2, n3, precision, &need));
  if (ws_bytes < need) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64)
    return tproj_run<double>((const double*)Q, (const double*)A, (const double*)dY, (double*)dQ, (double*)dA, n1, m,
                             n2, n3, ws, s);
  return tproj_run<float>((const float*)Q, (const float*)A, (const float*)dY, (float*)dQ, (float*)dA, n1, m, n2, n3,
                          ws, s);
}

extern "C" int tproj_workspace_size(int n1, int m, int n2, int n3, int precision, size_t* bytes) {
  return tproj_backward_workspace_size(n1, m, n2, n3, precision, bytes);
}

extern "C" int tproj(const void* Q, const void* A, void* Y, int n1, int m, int n2, int n3, int precision, void* ws,
                     size_t ws_bytes, void* stream) {
  if (!Q || !A || !Y || !ws || !dims_ok(n1, m, n2, n3) || !aligned(ws)) return TSVD_ERR_INVALID_ARG;
  size_t need;
  TSVD_TRY(tproj_workspace_size(n1, m, n2, n3, precision, &need));
  if (ws_bytes < need) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64)
    return tproj_fwd_run<double>((const double*)Q, (const double*)A, (double*)Y, n1, m, n2, n3, ws, s);
  return tproj_fwd_run<float>((const float*)Q, (const float*)A, (float*)Y, n1, m, n2, n3, ws, s);
}
