/*
 * tsvd.h -- C ABI of libtsvd: the randomized block Krylov truncated T-SVD
 * (Kooshkghazi, Ahmadi-Asl, de Almeida, "Randomized block Krylov method for
 * approximation of truncated tensor SVD", arXiv 2504.04989) and the t-product
 * with its adjoints, as hand-written CUDA kernels for one GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A real tensor X in R^{n1 x n2 x n3} is a dense row-major array of shape
 *    (n3, n1, n2): frontal slice t (Sec. 2, "frontal slices X^(k)") is
 *    contiguous, element X(i, j, t) sits at t*n1*n2 + i*n2 + j.
 *  - Element type: double for TSVD_FP64, float for every other precision.
 *  - Every pointer named "device" must point to memory of the current CUDA
 *    device (cudaMalloc'd or torch-allocated); the caller owns all memory.
 *    The library never allocates or frees memory on these paths: scratch space
 *    is the caller's workspace `ws` of at least the size the matching
 *    *_workspace_size call reports, aligned to 256 bytes.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on it; argument errors are reported synchronously as a
 *    negative return value and nothing is launched.
 *  - Results are deterministic for fixed inputs, parameters and seed (no
 *    atomics in reductions).
 *  - No C++ exception crosses this interface.
 */
#ifndef TSVD_H
#define TSVD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TSVD_API __attribute__((visibility("default")))
#else
#define TSVD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define TSVD_OK 0
#define TSVD_ERR_INVALID_ARG (-1)   /* null pointer, bad size, bad parameter, misaligned */
#define TSVD_ERR_WORKSPACE (-2)     /* ws_bytes smaller than required */
#define TSVD_ERR_CUDA (-3)          /* a CUDA launch or API call failed */
#define TSVD_ERR_UNSUPPORTED (-4)   /* size beyond a documented kernel limit */
#define TSVD_ERR_NOT_CONVERGED (-5) /* device side: an eigen solve did not converge */
#define TSVD_ERR_RANK_DEFICIENT (-6) /* device side: a Fourier slice of a pseudoinverse input lacks full rank */

/* ---- precision of the streaming contractions (FFT, Krylov, projection GEMMs) ---- */
typedef enum {
  TSVD_FP64 = 0,       /* everything in FP64 */
  TSVD_FP32 = 1,       /* FFT, complex GEMMs and the block orthonormalisation in FP32 (FP32
                          accumulation); the Gram of C and the small eigen-solve in FP64 */
  TSVD_MIXED_TF32 = 2, /* Krylov products on tcgen05 TF32, FP32 accumulation; rest as TSVD_FP32 */
  TSVD_MIXED_BF16 = 3, /* Krylov products on tcgen05 BF16, FP32 accumulation; rest as TSVD_FP32 */
  TSVD_SPLIT_TF32 = 4  /* tprod only: float arrays, the slice products on tcgen05 in split TF32
                          (x = hi + lo, hi*hi + hi*lo + lo*hi, operands carried to ~22 bits) */
} tsvd_precision;

/* ---- parameters of Alg. 2 (Sec. 3): target tubal rank R, oversampling P,
 *      power/Krylov depth q; seed of the Gaussian test tensor B = randn(n2, R+P, n3) ---- */
typedef struct {
  int R;
  int P;
  int q;
  int precision;  /* tsvd_precision */
  uint64_t seed;
  int flags;      /* bit 0 (TSVD_FLAG_FP64_QR): orthonormalise the Krylov blocks in FP64 on the
                     FP32 / mixed paths too (they use FP32 by default; the FP64 path always uses FP64);
                     bit 1 (TSVD_FLAG_ALG1): Alg. 1 instead of Alg. 2 */
} tsvd_params;

#define TSVD_FLAG_FP64_QR 1
/* bit 1 (TSVD_FLAG_ALG1): Alg. 1 of the paper (randomized subspace / power iteration):
   Q = orth((A A^H)^q A B), orthonormalised after every step (same span), basis of
   min(R+P, n1, n2) columns; the rest of the pipeline as for Alg. 2 */
#define TSVD_FLAG_ALG1 2
/* bit 2 (TSVD_FLAG_SIMT): FP32 / mixed paths: run the Krylov products on the FP32 SIMT units
   instead of the tensor cores (by default the FP32 path runs them on tcgen05 as split TF32,
   x = hi + lo with hi the nearest TF32, products hi*hi + hi*lo + lo*hi in FP32, about 22
   significant bits) */
#define TSVD_FLAG_SIMT 4
/* bit 3 (TSVD_FLAG_QTRUNC): Alg. 2 with the basis Q truncated to its leading R+P columns
   before the projection C = Q^T * X (the variant Sec. 5, Ex. 1 reports timings for); the
   Krylov steps still run in full.  m_eff then reports R+P. */
#define TSVD_FLAG_QTRUNC 8
/* bit 4 (TSVD_FLAG_DEFLATE, FP64 path only): deflated Rayleigh-Ritz passes in the small SVD.
   The Gram C C^H resolves singular values only down to ~1e-8 sigma_1; with this flag each
   pass keeps the eigenpairs with lambda >= 1e-6 lambda_max, projects them out of C and
   solves the rest again (six passes), so singular values down to the FP64 floor of C
   (absolute ~eps sigma_1) are returned, e.g. for the fast-decaying spectra of Sec. 5, Ex. 1.
   Other precisions return TSVD_ERR_UNSUPPORTED. */
#define TSVD_FLAG_DEFLATE 16
/* bit 5 (TSVD_FLAG_GRAM_INT, FP32 / mixed paths): take the exact Gram C C^H of the small SVD in
   64-bit integer multiply-adds on the SIMT units instead of its base-64 digit form on the BF16
   tensor cores (n2 <= 4096; larger n2 always use the integer form).  Both give the same G to
   the bit; the flag exists to compare them. */
#define TSVD_FLAG_GRAM_INT 32

/* ---- device-side outcome, read back only when requested ---- */
typedef struct {
  int status;          /* TSVD_OK or TSVD_ERR_NOT_CONVERGED */
  int m_eff;           /* basis columns per slice: min((q+1)(R+P), n1, n2) */
  int dead_columns;    /* Krylov columns found numerically dependent and replaced (all slices) */
  int reserved;
} tsvd_info;

/*
 * tsvd_rbk_workspace_size -- bytes of workspace tsvd_rbk needs for this shape.
 * Returns TSVD_OK and writes *bytes, or TSVD_ERR_INVALID_ARG / TSVD_ERR_UNSUPPORTED.
 */
TSVD_API int tsvd_rbk_workspace_size(int n1, int n2, int n3, const tsvd_params* params, size_t* bytes);

/*
 * tsvd_rbk -- randomized block Krylov truncated T-SVD, Alg. 2 of the paper
 * (Sec. 3), computed slice by slice in the Fourier domain (the remark opening
 * Sec. 4; Alg. TP / Alg. TQR for the transform and the mirror).
 *
 *   A      device, (n3, n1, n2) real, the data tensor X.
 *   params R >= 1, R <= min(n1, n2), P >= 0, q >= 0; precision; seed.
 *   Omega  device, (n3, n2, R+P) real test tensor B of Alg. 2, or NULL to draw
 *          it on the device: element e is output e%4 of Philox4x32-10 call e/4
 *          with counter (e/4 low, e/4 high, 0, 0) and key (seed low, seed high);
 *          words (x0,x1) and (x2,x3) become normals by Box-Muller with
 *          uniforms (x+1)/2^32: r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2).
 *   U      device out, (n3, n1, R): U_R of Alg. 2 (last line).
 *   S      device out, (n3, R): the diagonal tubes of the f-diagonal S_R.
 *   V      device out, (n3, n2, R): V_R.
 *   sigma_hat  device out (double), (floor(n3/2)+1, R): Fourier-domain singular
 *          values per slice, descending; may be NULL.
 *   ws, ws_bytes  device workspace (see tsvd_rbk_workspace_size).
 *   info   host out, may be NULL.  When non-NULL the call synchronises `stream`
 *          and fills it; otherwise the call is fully asynchronous.
 * Limits: R + P <= 128, min((q+1)(R+P), n1, n2) <= 512 (TSVD_ERR_UNSUPPORTED).
 * The Krylov block is built in its block-orthonormalised form (same span as
 * K = [K_0..K_q] in exact arithmetic): Q_0 = orth(A B), Q_i = orth(A A^H Q_{i-1}
 * minus its part in Q_0..Q_{i-1}); the last block keeps its leading columns.
 */
TSVD_API int tsvd_rbk(const void* A, int n1, int n2, int n3, const tsvd_params* params, const void* Omega,
             void* U, void* S, void* V, double* sigma_hat, void* ws, size_t ws_bytes, void* stream,
             tsvd_info* info);

/*
 * tsvd_rbk_batched -- Alg. 2 on a batch of independent tensors of different
 * shapes, ranks and parameters (the slices of every tensor, and the tensors
 * themselves, are independent problems: the remark opening Sec. 4).
 *
 *   descs  host array of `count` descriptors: each names one tsvd_rbk call
 *          (A, n1, n2, n3, params, Omega, U, S, V, sigma_hat with tsvd_rbk's
 *          meaning, layouts and limits; device pointers; sigma_hat and Omega
 *          may be NULL).  The library reads the array during the call only.
 *   lanes  number of concurrent CUDA streams (1..32; more than `count` is
 *          clamped).  Tensors are ordered by an estimate of their work
 *          (largest first) and each goes to the lane with the least work so
 *          far; a lane runs its tensors in that order.
 *   ws, ws_bytes  device workspace of tsvd_rbk_batched_workspace_size bytes
 *          for the same descriptors and lanes (the sum over lanes of the
 *          largest tsvd_rbk workspace among the lane's tensors).
 *   stream the caller's stream: the lanes start after the work already
 *          queued on it and it waits for all of them at the end, so the call
 *          is asynchronous and can be captured into a CUDA graph (the first
 *          call on a device creates the lane streams and events, so make one
 *          call before capturing).
 * The lane streams are shared by all calls on a device: calls whose work
 * overlaps in time (different host threads or unordered streams) must not be
 * issued concurrently.  Results equal those of separate tsvd_rbk calls.
 */
typedef struct {
  const void* A;
  int n1, n2, n3;
  tsvd_params params;
  const void* Omega;
  void* U;
  void* S;
  void* V;
  double* sigma_hat;
} tsvd_rbk_desc;

TSVD_API int tsvd_rbk_batched_workspace_size(const tsvd_rbk_desc* descs, int count, int lanes, size_t* bytes);
TSVD_API int tsvd_rbk_batched(const tsvd_rbk_desc* descs, int count, int lanes, void* ws, size_t ws_bytes,
                              void* stream);

/*
 * tprod -- t-product C = A * B (Definition of the T-product, Sec. 2, computed
 * by Alg. TP: mode-3 FFT, one complex product per non-redundant Fourier slice,
 * conjugate mirror, inverse FFT).
 *   A device (n3, n1, n2), B device (n3, n2, n4), C device out (n3, n1, n4).
 *   precision: TSVD_FP64 (double arrays) or TSVD_FP32 / TSVD_MIXED_TF32 /
 *   TSVD_MIXED_BF16 (float arrays; the slice products on FP32 SIMT or tcgen05).
 */
TSVD_API int tprod_workspace_size(int n1, int n2, int n4, int n3, int precision, size_t* bytes);
TSVD_API int tprod(const void* A, const void* B, void* C, int n1, int n2, int n4, int n3, int precision, void* ws,
          size_t ws_bytes, void* stream);

/*
 * tproj -- projection Y = Q * Q^T * A onto the range of Q (the projector of
 * the Sec. 4 lemma A - U_k * U_k^T * A = A - Q * (Q^T * A)_k), per Fourier
 * slice Y_k = Q_k (Q_k^H A_k).
 *   Q device (n3, n1, m), A device (n3, n1, n2), Y device out (n3, n1, n2).
 */
TSVD_API int tproj_workspace_size(int n1, int m, int n2, int n3, int precision, size_t* bytes);
TSVD_API int tproj(const void* Q, const void* A, void* Y, int n1, int m, int n2, int n3, int precision, void* ws,
                   size_t ws_bytes, void* stream);

/*
 * tprod_backward -- adjoint of the t-product for L = <dC, A*B> (inner product
 * of Sec. 2): dA = dC * B^T and dB = A^T * dC, with the tensor transpose of
 * Sec. 2 (bcirc(X^T) = bcirc(X)^T).  In the Fourier domain these are
 * dA_k = dC_k B_k^H and dB_k = A_k^H dC_k.  Either output may be NULL.
 *   A (n3,n1,n2), B (n3,n2,n4), dC (n3,n1,n4); dA (n3,n1,n2), dB (n3,n2,n4).
 */
TSVD_API int tprod_backward_workspace_size(int n1, int n2, int n4, int n3, int precision, size_t* bytes);
TSVD_API int tprod_backward(const void* A, const void* B, const void* dC, void* dA, void* dB, int n1, int n2, int n4,
                   int n3, int precision, void* ws, size_t ws_bytes, void* stream);

/*
 * tproj_backward -- adjoint of the projection Y = Q * Q^T * A (the projector
 * of the Sec. 4 lemma): dA = Q * (Q^T * dY) and
 * dQ = dY * (A^T * Q) + A * (dY^T * Q).
 *   Q (n3,n1,m), A (n3,n1,n2), dY (n3,n1,n2); dQ (n3,n1,m), dA (n3,n1,n2).
 *   Either output may be NULL.
 */
TSVD_API int tproj_backward_workspace_size(int n1, int m, int n2, int n3, int precision, size_t* bytes);
TSVD_API int tproj_backward(const void* Q, const void* A, const void* dY, void* dQ, void* dA, int n1, int m, int n2, int n3,
                   int precision, void* ws, size_t ws_bytes, void* stream);

/*
 * ttranspose -- tensor transpose (Sec. 2, Definition of the transpose):
 * AT(:,:,1) = A(:,:,1)^T and AT(:,:,k) = A(:,:,n3+2-k)^T for k = 2..n3 (1-based).
 *   A device (n3, n1, n2), AT device out (n3, n2, n1); double for TSVD_FP64,
 *   float otherwise.  Out of place (A and AT must not overlap).
 */
TSVD_API int ttranspose(const void* A, void* AT, int n1, int n2, int n3, int precision, void* stream);

/*
 * tsvd_masked_residual -- residual of the completion objective
 * ||P_Omega(C) - P_Omega(X)||_F^2 (the observation operator of Ex. 3):
 *   R = M .* (C - X) element-wise and *loss = sum(R^2) (FP64, device).
 *   C, X, R device arrays of n elements (double for TSVD_FP64, float
 *   otherwise); mask device uint8 (nonzero = observed); partial device
 *   scratch of 1024 doubles.  The sum is reduced in a fixed order.
 */
TSVD_API int tsvd_masked_residual(const void* C, const void* X, const uint8_t* mask, void* R, double* loss,
                                  double* partial, long n, int precision, void* stream);

/*
 * tsvd_error -- squared approximation error ||X - U * S * V^T||_F^2 of a
 * truncated T-SVD (the error measure of the experiments, Sec. 5), evaluated
 * in the Fourier domain: Parseval (Sec. 2) over the floor(n3/2)+1 leading
 * Fourier slices with weight 1 for slice 0 and slice n3/2 (n3 even) and 2 for
 * the rest, one fused pass per slice that forms X_k - U_k diag(s_k) V_k^H
 * tile by tile and accumulates only its squared modulus (FP64).
 *   X device (n3, n1, n2); U device (n3, n1, R); S device (n3, R) diagonal
 *   tubes of the f-diagonal S; V device (n3, n2, R) (tsvd_rbk's layouts).
 *   err2   device out, one double.
 *   precision TSVD_FP64 (double arrays, FP64 arithmetic) or any other
 *   (float arrays; FP32 products, FP64 accumulation of the squares).
 *   ws, ws_bytes  device workspace of tsvd_error_workspace_size bytes.
 */
TSVD_API int tsvd_error_workspace_size(int n1, int n2, int n3, int R, int precision, size_t* bytes);
TSVD_API int tsvd_error(const void* X, const void* U, const void* S, const void* V, int n1, int n2, int n3, int R,
                        int precision, double* err2, void* ws, size_t ws_bytes, void* stream);

/*
 * tsvd_rfft3 / tsvd_irfft3 -- the mode-3 transforms of the method (Sec. 2,
 * Def. of F_n: unnormalised forward DFT along the third mode, omega =
 * e^{-2 pi i / n3}; the inverse scaled by 1/n3 after the conjugate mirror of
 * Alg. TP).  X device (n3, plane) real, a tensor (n3, rows, cols) with
 * plane = rows * cols; Xhat device (floor(n3/2)+1, plane) complex
 * interleaved.  precision TSVD_FP64 (double) or TSVD_FP32 (float).
 */
TSVD_API int tsvd_rfft3(const void* X, long plane, int n3, int precision, void* Xhat, void* stream);
TSVD_API int tsvd_irfft3(const void* Xhat, long plane, int n3, int precision, void* X, void* stream);

/*
 * tsvd_rbk_fourier -- Alg. 2 (Sec. 3) on the block of Fourier slices
 * [k0, k0 + ns) of an n1 x n2 x n3 tensor whose half spectrum the caller
 * already holds (the remark opening Sec. 4: the slices are independent
 * problems).  This is the per-device step of the slice-sharded multi-GPU
 * path.  Every slice sees the same test tensor as tsvd_rbk: the real Omega
 * (n3, n2, R+P) is drawn (or taken from Omega) and transformed whole.
 *   Ahat device (ns, n1, n2) complex (double2 for FP64, float2 otherwise),
 *   slice k0 + s at index s; outputs in the Fourier domain: Uhat device
 *   (ns, n1, R), Vhat device (ns, n2, R) in Ahat's complex type, sigma_hat
 *   device (ns, R) double.  params, workspace, stream and info as tsvd_rbk.
 *   0 <= k0, ns >= 1, k0 + ns <= floor(n3/2)+1, else TSVD_ERR_INVALID_ARG.
 */
TSVD_API int tsvd_rbk_fourier_workspace_size(int n1, int n2, int n3, int k0, int ns, const tsvd_params* params,
                                             size_t* bytes);
TSVD_API int tsvd_rbk_fourier(const void* Ahat, int n1, int n2, int n3, int k0, int ns, const tsvd_params* params,
                              const void* Omega, void* Uhat, void* Vhat, double* sigma_hat, void* ws, size_t ws_bytes,
                              void* stream, tsvd_info* info);

/*
 * Data completion of Sec. 5, Ex. 3: the iteration X^(n) = L(C^(n)) (L the
 * truncated T-SVD of Alg. 2 followed by the product below) and
 * C^(n+1) = T .* M + (1 - T) .* X^(n), T the observation mask, M the data.
 *
 * tsvd_lowrank -- X = U * S * V^T from the spatial factors of tsvd_rbk:
 *   U (n3, n1, R), S (n3, R) singular tubes, V (n3, n2, R); X out (n3, n1, n2);
 *   per Fourier slice X_k = U_k diag(S_k) V_k^H (Alg. TP), then the inverse
 *   transform.  FP64 or FP32; workspace from tsvd_lowrank_workspace_size.
 * tsvd_sigma_tubes -- the f-diagonal tubes of S^power (power 1 or 1/2, any
 *   positive power accepted) from the Fourier-domain singular values
 *   sigma_hat (floor(n3/2)+1, R): tubes out (n3, R); ws holds
 *   (floor(n3/2)+1) * R complex elements (16 or 8 bytes each).
 * tsvd_fill_in -- C <- mask ? M : X element-wise over n elements (mask bytes
 *   nonzero = observed) and *change2 = sum (C_new - C_old)^2 in FP64 (device
 *   scalar); partial is a device scratch of 1024 doubles.
 * tsvd_sqdiff -- *out = sum (A - B)^2 over n elements in FP64 (device scalar),
 *   the squared error behind PSNR = 10 log10(peak^2 n / sum); partial as above.
 * All are asynchronous on `stream`; argument errors return at once.
 */
TSVD_API int tsvd_lowrank_workspace_size(int n1, int n2, int n3, int R, int precision, size_t* bytes);
TSVD_API int tsvd_lowrank(const void* U, const void* S, const void* V, int n1, int n2, int n3, int R, int precision,
                          void* X, void* ws, size_t ws_bytes, void* stream);
TSVD_API int tsvd_sigma_tubes(const double* sigma_hat, int R, int n3, double power, int precision, void* tubes,
                              void* ws, size_t ws_bytes, void* stream);
TSVD_API int tsvd_fill_in(void* C, const void* M, const uint8_t* mask, const void* X, long n, int precision,
                          double* partial, double* change2, void* stream);
TSVD_API int tsvd_sqdiff(const void* A, const void* B, long n, int precision, double* partial, double* out,
                         void* stream);

/*
 * tqr -- T-QR decomposition X = Q * R (Alg. TQR, Sec. 2): per non-redundant
 * Fourier slice the economy QR of X_k with p = min(n1, n2), the other slices
 * by conjugate symmetry, and the inverse transform of both factors.  The QR of
 * a slice is unique up to unit phases on the diagonal of R; this library
 * returns the factors whose Fourier slices have diag(R_k) real and >= 0.  A
 * slice wider than tall is factored on its first n1 columns (R = Q^H X).
 *   A device (n3, n1, n2) real; Q device out (n3, n1, p); R device out
 *   (n3, p, n2); precision TSVD_FP64 (double) or TSVD_FP32 (float).
 *   Workspace from tqr_workspace_size, 256-byte aligned.  Numerically
 *   dependent columns are replaced by orthonormal directions (Q keeps
 *   orthonormal columns; R has ~0 on those diagonal entries); their number is
 *   returned in info->dead_columns when info is non-NULL (synchronises).
 */
TSVD_API int tqr_workspace_size(int n1, int n2, int n3, int precision, size_t* bytes);
TSVD_API int tqr(const void* A, int n1, int n2, int n3, int precision, void* Q, void* R, void* ws, size_t ws_bytes,
                 void* stream, tsvd_info* info);

/*
 * tpinv -- Moore-Penrose pseudoinverse X^+ (Alg. mp, Sec. 2): per Fourier
 * slice pinv(X_k), computed as R_k^{-1} Q_k^H from the QR of X_k (n1 >= n2) or
 * of X_k^H (n1 < n2, pinv(X) = pinv(X^H)^H), then the inverse transform.  It
 * equals the pseudoinverse when every Fourier slice has full rank
 * min(n1, n2); a rank-deficient slice sets info->status to
 * TSVD_ERR_RANK_DEFICIENT (info non-NULL: the call synchronises) and the
 * output is then not the pseudoinverse.
 *   A device (n3, n1, n2) real; X device out (n3, n2, n1); precision FP64 / FP32.
 */
TSVD_API int tpinv_workspace_size(int n1, int n2, int n3, int precision, size_t* bytes);
TSVD_API int tpinv(const void* A, int n1, int n2, int n3, int precision, void* X, void* ws, size_t ws_bytes,
                   void* stream, tsvd_info* info);

/*
 * tprod_noalloc -- the t-product C = A * B of tprod(), for callers that cannot
 * allocate device memory (an arena or pool that must not grow, a plug-in whose
 * host process owns every device allocation, a real-time loop where an
 * allocation would stall).  The paper has no counterpart: this is a service of
 * the library.  It takes no workspace: its scratch is a fixed 16 MiB array
 * inside the library (reserved on every GPU that loads the library until the
 * process exits), and it calls no allocating routine.
 *   A device (n3, n1, n2), B device (n3, n2, n4), C device out (n3, n1, n4);
 *   precision TSVD_FP64 (double) or TSVD_FP32 (float).
 * Limit: the three half-spectrum operands, (floor(n3/2)+1) * (n1*n2 + n2*n4 +
 * n1*n4) complex elements (8 bytes each in FP32, 16 in FP64, each array rounded
 * up to 256 bytes), must fit in 16 MiB; larger problems return
 * TSVD_ERR_UNSUPPORTED and launch nothing.
 * All calls share the array: calls whose kernels overlap on the GPU race.
 * The array sits in a module of the library that holds no kernel; with CUDA's
 * lazy module loading (the default) that module, and its 16 MiB, is loaded on
 * a device by the first call there, so make that first call before sealing a
 * pool that must not grow and before capturing a CUDA graph.  Every call
 * outside a capture looks the array's address up again (nothing is allocated
 * by that once the module is loaded), so a device reset is followed; inside a
 * capture the address from the last uncaptured call on the device is used
 * (TSVD_ERR_CUDA if there was none).
 */
TSVD_API int tprod_noalloc(const void* A, const void* B, void* C, int n1, int n2, int n4, int n3, int precision,
                           void* stream);

/* Philox4x32-10 Gaussian draw of the test tensor on the device (the same
 * definition as tsvd_rbk uses when Omega is NULL), for inspection and tests:
 * out (device, double) receives n normals of (seed, stream, tensor_id). */
TSVD_API int tsvd_gaussian(uint64_t seed, uint32_t stream_id, uint32_t tensor_id, long n, double* out, void* stream);
/* raw Philox words for counters ctr0..ctr0+n-1 (ctr1..3 fixed), 4 words each */
TSVD_API int tsvd_philox_words(const uint32_t key[2], uint32_t ctr1, uint32_t ctr2, uint32_t ctr3, long n, uint32_t* out,
                      void* stream);

/* ---- optional stage timing (diagnostic, process-global, not thread safe) ----
 * Between tsvd_profile_begin() and tsvd_profile_end() every pipeline stage of
 * the calls above records a CUDA event pair on its stream.  tsvd_profile_end()
 * synchronises those events and writes up to max_out per-stage totals
 * (summed milliseconds and the number of recorded stage executions); *n_out
 * receives the number written. */
typedef struct {
  char name[32];
  double ms;
  int count;
} tsvd_stage_time;
TSVD_API int tsvd_profile_begin(void);
TSVD_API int tsvd_profile_end(tsvd_stage_time* out, int max_out, int* n_out);

/* number of kernels the library has launched in this process (all threads) */
TSVD_API unsigned long long tsvd_launch_count(void);

TSVD_API const char* tsvd_strerror(int code);
/* library version (major*10000 + minor*100 + patch) */
TSVD_API int tsvd_version(void);

#ifdef __cplusplus
}
#endif
#endif
