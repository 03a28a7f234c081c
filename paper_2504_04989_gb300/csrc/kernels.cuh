// kernels.cuh -- host launchers shared between the translation units of libtsvd.
#pragma once

#include "common.cuh"

namespace tsvd {

// RAII stage timer: records a CUDA event pair around a pipeline stage when
// stage profiling is enabled (profile.cu); no-op otherwise.
class StageTimer {
 public:
  StageTimer(const char* name, cudaStream_t s);
  ~StageTimer();

 private:
  const char* name_;
  cudaStream_t s_;
  void* a_;
};
#define TSVD_CAT2(a, b) a##b
#define TSVD_CAT(a, b) TSVD_CAT2(a, b)
#define TSVD_STAGE(name, s) ::tsvd::StageTimer TSVD_CAT(_stage_timer_, __LINE__)(name, s)

// fft.cu
template <typename T>
int launch_rfft3(const T* X, cx_t<T>* Xh, long plane, int n3, cudaStream_t s);
template <typename T>
int launch_irfft3(const cx_t<T>* Xh, T* X, long plane, int n3, cudaStream_t s);
template <typename T>
int launch_gaussian(uint64_t seed, uint32_t stream_id, uint32_t tensor_id, long n, T* out, cudaStream_t s);

// cgemm.cu -- batched complex GEMM on the SIMT pipes,
//   C_b = alpha * op(A_b) * op(B_b) + beta * C_b   for b < batch,
// op = 'N' (as stored) or 'H' (conjugate transpose); all row-major.
// op(A) is M x K, op(B) is K x N; C is M x N with leading dimension ldc.
// beta must be 0 or 1 (C is not read when beta == 0).  When ksplit > 1 the K
// range is split over CTAs; `splitk_ws` must hold ksplit*batch*M*N elements.
struct GemmArgs {
  char opA, opB;
  int M, N, K;
  double alpha, beta;
  const void* A;
  long lda, sA;
  const void* B;
  long ldb, sB;
  void* C;
  long ldc, sC;
  int batch;
};
// GemmArgs from its fields (strided batch)
inline GemmArgs gemm(char opA, char opB, int M, int N, int K, double alpha, const void* A, long lda, long sA,
                     const void* B, long ldb, long sB, double beta, void* Cm, long ldc, long sC, int batch) {
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
  g.sA = sA;
  g.B = B;
  g.ldb = ldb;
  g.sB = sB;
  g.C = Cm;
  g.ldc = ldc;
  g.sC = sC;
  g.batch = batch;
  return g;
}
template <typename C>
int cgemm(const GemmArgs& g, void* splitk_ws, size_t splitk_elems, cudaStream_t s);
// C = op(A) op(B) known to be Hermitian (square, beta = 0, e.g. A^H A): only
// the upper tiles are computed, the lower triangle is mirrored from them
template <typename C>
int cgemm_herm(const GemmArgs& g, void* splitk_ws, size_t splitk_elems, cudaStream_t s);
// pick a split of K that fills the GPU (bounded by the scratch it needs)
int choose_ksplit(int M, int N, int K, int batch, size_t splitk_elems);

// element-wise conversions of batched complex matrices (rows x cols, leading dims)
int convert_c64_to_c32(const double2* src, long lds, long ss, float2* dst, long ldd, long sd, int rows, int cols,
                       int batch, cudaStream_t s);
int convert_c32_to_c64(const float2* src, long lds, long ss, double2* dst, long ldd, long sd, int rows, int cols,
                       int batch, cudaStream_t s);
template <typename C>
int copy_cx(const C* src, long lds, long ss, C* dst, long ldd, long sd, int rows, int cols, int batch,
            cudaStream_t s);

// cholqr.cu -- block orthonormalisation pieces (one problem per Fourier slice)
// Cholesky R^H R = G + s I of the nb x nb Hermitian Gram G (s = shift_rel *
// trace(G) when shift_rel > 0) in G's precision, then M = R-tilde^{-1} written
// dense (zeros below the diagonal) in the same precision.  Pivots: shifted
// pass -> dead iff d_j <= 0; plain pass -> dead iff d_j <= dead_rel * G_jj.
// Dead columns are marked in `dead` (4 words per slice); R-tilde has unit
// rows and columns there and M zero columns, so W M = W_live R_live^{-1} on
// the live columns and 0 on the dead ones.
template <typename GC>
int chol_inv(const GC* G, long ldg, long sG, GC* M, long ldm, long sM, int nb, int batch, double shift_rel,
             double dead_rel, uint32_t* dead, cudaStream_t s);
// O <- W M for the n1 x nb blocks of every slice (M nb x nb dense); O may be W itself (each CTA
// stages its rows of W before writing).
template <typename C>
int rmul_block(const C* W, long ldw, long sW, const C* M, long ldm, long sM, int n1, int nb, int batch, C* O, long ldo,
               long sO, cudaStream_t s);
// Replace dead columns [c, c+nb) of Q (n1 x ldq per slice) by unit vectors
// orthogonal to columns [0, c+nb): Philox directions projected twice.  Problem
// b is Fourier slice k0 + b; slice 0 and slice nyq (n3/2 for an even n3, else
// -1) get real directions, as the spectrum of a real tensor is real there.
template <typename C>
int repair_dead(C* Q, long ldq, long sQ, int n1, int c, int nb, const uint32_t* dead, int batch, uint64_t seed,
                int block_id, int* dead_count, int k0, int nyq, cudaStream_t s);
// Block orthonormalisation step of a basis Q (n1 x m per slice, leading dim m)
// in precision L: the nb leading columns of W (n1 x b, leading dim b) are made
// orthonormal against Q's c finished columns by shifted CholeskyQR3 with a
// classical Gram-Schmidt projection before each pass, written to Q columns
// [c, c + nb); dependent columns are replaced (repair_dead, counted in
// *dead_count).  P (m x b), G and Minv (b x b) are scratch; when Qt is set the
// block is also converted to FP32 there (L = double with FP32 GEMM data).
// Split-TF32 tensor-core operands of the FP32 block orthonormalisation (its
// block Gram and W R^-1 on tcgen05 instead of the SIMT GEMMs); per slice:
struct OrthTc {
  float *WThi, *WTlo;  // W^T: b rows of 2 n1 floats (leading dim ldq2)
  float *Whi, *Wlo;    // W as real rows: n1 rows of 2 b floats (leading dim ldw2)
  float *Ehi, *Elo;    // expanded real forms of the thin factors: 2b rows (leading dim <= ldq2)
  float *Qhi, *Qlo;    // finished basis columns as real rows: n1 rows of 2 m floats (leading dim ldqi)
  float *Qdhi, *Qdlo;  // ... and de-interleaved: 2m rows of n1 floats (leading dim ldq2 / 2)
  long ldq2, ldw2, ldqi;
  int* err;            // set by a tcgen05 pipeline wait that timed out
};

struct OrthWs {
  void* Q;
  void* W;
  void* P;
  void* G;
  void* Minv;
  uint32_t* dead;
  int* dead_count;
  void* Qt;
  void* splitk;
  size_t splitk_elems;  // in double2 elements
  int k0;               // Fourier slice index of problem 0
  int nyq;              // index of the (real) Nyquist slice, n3/2 for an even n3, else -1
  const OrthTc* tc;     // FP32: products on tcgen05 (split TF32), or nullptr for the SIMT GEMMs
};
template <typename L>
int orth_block_cols(int n1, int b, int m, int h, const OrthWs& w, int c, int nb, int block_id, uint64_t seed,
                    cudaStream_t s);
// tc_gemm.cu -- tcgen05 tensor-core GEMM C_b (M x N, FP32) = A_b (M x K) B_b^T
// with A (M x K) and B (N x K) K-major, TF32 (FP32 storage) or BF16.  Needs
// 16-byte aligned bases, row strides and batch strides (tc_gemm_supported);
// *err is set if a pipeline wait timed out.
bool tc_gemm_supported(const void* A, long lda, long sA, const void* B, long ldb, long sB, int batch, bool bf16);
// upper: a symmetric product (B = A, M = N): only the tiles not wholly below the diagonal are
// written (tile rows of 128, tile columns of tc_gemm_tile_n(N, bf16))
int tc_gemm(const void* A, long lda, long sA, int M, const void* B, long ldb, long sB, int N, int K, float* C, long ldc,
            long sC, int batch, bool bf16, int* err, cudaStream_t s, bool upper = false);
int tc_gemm_tile_n(int N, bool bf16);
// expanded real form E (2N x 2K, leading dim lde) of a thin interleaved complex
// Y (K x N): real(X) E^T = X Y (mode 0) or conj(X) Y (mode 1)
int expand_thin(const float2* Y, long ldy, long sy, int K, int N, void* E, long lde, long se, int batch, int mode,
                bool bf16, cudaStream_t s);
// rows x cols FP32 rows (leading dim ldx) copied to BF16 or FP32 rows of leading dim ldy (zero padded)
int copy_rows(const float* x, long ldx, void* y, long ldy, int cols, long rows, bool bf16, cudaStream_t s);
// split TF32: C = alpha A B^T + beta C with A = Ahi + Alo, B = Bhi + Blo (hi*hi + hi*lo + lo*hi),
// FP32-level accuracy
// Optional split copies of the result written by the epilogue (null pointers: none):
//   rows (Rhi / Rlo): hi / lo of C in C's own layout (leading dim ldr, batch stride sr);
//   cols (Thi / Tlo): hi / lo of C^T (row f of T is column f of C; leading dim ldt, batch stride st).
struct TcSplitOut {
  float *Rhi = nullptr, *Rlo = nullptr;
  long ldr = 0, sr = 0;
  float *Thi = nullptr, *Tlo = nullptr;
  long ldt = 0, st = 0;
};
int tc_gemm_split(const float* Ahi, const float* Alo, long lda, long sA, int M, const float* Bhi, const float* Blo,
                  long ldb, long sB, int N, int K, float* C, long ldc, long sC, int batch, int* err, cudaStream_t s,
                  float alpha = 1.0f, float beta = 0.0f, const TcSplitOut* out2 = nullptr);
// FP32 rows -> hi (nearest TF32) / lo rows of leading dim ldy, padding zeroed
int split_rows(const float* x, long ldx, float* hi, float* lo, long ldy, int cols, long rows, cudaStream_t s);
// columns [0, cols) of FP32 rows -> hi / lo rows (leading dim ldy); other columns untouched
int split_block(const float* x, long ldx, float* hi, float* lo, long ldy, int cols, long rows, cudaStream_t s);
// per slice complex X (rows x cols) -> X^T as real rows of 2 rows floats (leading dim ldt), hi / lo
int split_transpose(const float2* X, int rows, int cols, int batch, float* hi, float* lo, long ldt, cudaStream_t s);
// the same for a strided block (leading dim ldx, batch stride sx) into rows of leading dim ldt, batch stride st
// (padding columns are not touched)
int split_transpose_ld(const float2* X, int rows, int cols, long ldx, long sx, int batch, float* hi, float* lo,
                       long ldt, long st, cudaStream_t s);
// per slice the columns c of a complex X (rows x cols, leading dim ldx, batch stride sx) as real
// rows 2c (real parts) and 2c+1 (imaginary parts) of length rows, split into hi / lo (leading dim
// ldt, batch stride st; padding not touched)
int split_deinterleave(const float2* X, int rows, int cols, long ldx, long sx, int batch, float* hi, float* lo,
                       long ldt, long st, cudaStream_t s);
// expand_thin into FP32 hi / lo parts
int expand_thin_split(const float2* Y, long ldy, long sy, int K, int N, float* Eh, float* El, long lde, long se,
                      int batch, int mode, cudaStream_t s);
// eig.cu
// Eigen-decomposition of the m x m Hermitian G per slice (G is overwritten):
// top-R eigenvalues (descending) in lam (batch x R) and eigenvectors in
// U (batch x m x R, row-major, leading dim ldu) in U's precision.
size_t eig_scratch_bytes(int m, int R, int batch);
template <typename C>
int herm_eig_topR(double2* G, long ldg, long sG, int m, int R, int batch, double* lam, C* U, long ldu, long sU,
                  void* scratch, int* status, cudaStream_t s);
// sigma = sqrt(max(lam, 0)) -> sig (batch x R, may be null) and the complex
// tube slices Sh of S; a non-finite eigenvalue sets *status.
template <typename T>
int sigma_from_lambda(const double* lam, int R, int batch, double* sig, cx_t<T>* Sh, cudaStream_t s, int* status);
// columns r of V (rows x R per slice) scaled by 1 / sqrt(lam_r) (zero where lam_r <= 0)
template <typename T>
int scale_columns_inv(cx_t<T>* V, long ldv, long sV, int rows, int R, const double* lam, int batch, cudaStream_t s);

// deflate.cu -- one merge step of the deflated Rayleigh-Ritz passes: the
// pass's eigenpairs with lambda >= 1e-6 lambda_max (all missing ones when
// `last`) are appended per slice to lamF (batch x R) and UF, Um (batch x mp x
// R; Um keeps zeros beyond the accepted columns); acc (batch) counts them.
int deflate_merge(const double* lam_p, const double2* U_p, int mp, int R, int batch, double* lamF, double2* UF,
                  double2* Um, int* acc, bool first, bool last, cudaStream_t s);

// gram_int.cu -- G = C C^H (Hermitian, FP64 out) from FP32 C^H (n2 x m per
// slice, leading dimension ldc): per-column power-of-two scaling to integers
// and an exact 64-bit integer Gram.  Q (batch x n2 x m int2) and colexp
// (batch x m) are scratch.
int gram_int_fp32(const float2* CH, long ldc, long sC, int n2, int m, int batch, int2* Q, int* colexp, double2* G,
                  long ldg, long sG, cudaStream_t s);
// the same G, bitwise, from base-64 digits of the integers on the BF16 tensor cores (n2 <= 4096):
// gram_sliced_bytes of scratch in ws, colexp (batch x m) as above; err as for tc_gemm
bool gram_sliced_ok(int n2, int m);
size_t gram_sliced_bytes(int n2, int m, int batch);
int gram_sliced_fp32(const float2* CH, long ldc, long sC, int n2, int m, int batch, int* colexp, void* ws,
                     double2* G, long ldg, long sG, int* err, cudaStream_t s);

}  // namespace tsvd
