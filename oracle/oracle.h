/*
 * oracle.h -- plain FP64 CPU oracle for the randomized block Krylov truncated
 * T-SVD (Kooshkghazi, Ahmadi-Asl, de Almeida, arXiv 2504.04989).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test suite, the smoke check in __graft_entry__ and the cpu_baseline leg of
 * bench.py may load it.  It shares no code, header, table or helper with the
 * CUDA path under paper_2504_04989_gb300/.
 *
 * Conventions (all arrays row-major, caller-allocated):
 *   real tensor X in R^{n1 x n2 x n3}: frontal slice t is contiguous,
 *       element X(i,j,t) at  t*n1*n2 + i*n2 + j      (shape (n3, n1, n2))
 *   half spectrum (Sec. 2, Alg. TP): h = floor(n3/2)+1 = ceil((n3+1)/2) slices,
 *       complex interleaved, slice k element (i,j) at k*n1*n2 + i*n2 + j
 *   complex = two doubles (re, im), i.e. C99 double complex.
 *
 * Every function returns 0 on success and a negative value on a bad argument.
 */
#ifndef TSVD_ORACLE_H
#define TSVD_ORACLE_H

#include <complex.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef double complex orc_cplx;

/* ---- counter-based Gaussian draw (reading of randn in Alg. 1 / Alg. 2) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* n standard normals for elements 0..n-1 of stream `stream` of tensor `tensor_id`. */
void orc_gaussian(uint64_t seed, uint32_t stream, uint32_t tensor_id, long n, double* out);

/* ---- mode-3 DFT (Sec. 2, Def. of F_n; Alg. TP first lines) ---- */
int orc_dft_mode3(const double* X, int n1, int n2, int n3, const int* slices, int ns, orc_cplx* Xhat);
/* inverse from the half spectrum: conjugate mirror (Alg. TP) then F^{-1} = F^* / n */
int orc_idft_mode3(const orc_cplx* Xhat, int n1, int n2, int n3, double* X);

/* ---- t-algebra (Sec. 2) ---- */
int orc_tprod(const double* A, const double* B, int n1, int n2, int n4, int n3, double* C);        /* Alg. TP */
int orc_tprod_bcirc(const double* A, const double* B, int n1, int n2, int n4, int n3, double* C);  /* Def. fold(bcirc(A) unfold(B)) */
int orc_ttranspose(const double* A, int n1, int n2, int n3, double* AT);                           /* Def. tensor transpose */
int orc_tprod_backward(const double* A, const double* B, const double* dC, int n1, int n2, int n4, int n3,
                       double* dA, double* dB);
int orc_tproj_backward(const double* Q, const double* A, const double* dY, int n1, int m, int n2, int n3,
                       double* dQ, double* dA);

/* ---- dense per-slice linear algebra ---- */
/* economy Householder QR of an M x N complex matrix (M >= N): Q is M x N with orthonormal columns */
int orc_householder_qr(int M, int N, const orc_cplx* X, orc_cplx* Q, orc_cplx* Rf);
/* one-sided (Hestenes) Jacobi SVD of an M x N complex matrix, M >= N:
 * X = W diag(s) V^H, s descending, W M x N, V N x N unitary.  Returns sweeps used (>0) or <0 */
int orc_jacobi_svd(int M, int N, const orc_cplx* X, orc_cplx* W, double* s, orc_cplx* V);

/* ---- randomized T-SVD in the Fourier domain (Sec. 3) ---- */
/* ORC_ALG2_QTRUNC: Alg. 2 with the basis Q truncated to its leading R+P
 * columns before the projection (the variant Ex. 1 of Sec. 5 reports). */
enum { ORC_ALG2_CANONICAL = 0, ORC_ALG2_LITERAL = 1, ORC_ALG1_POWER = 2, ORC_EXACT = 3, ORC_ALG2_QTRUNC = 4 };
/*
 * For every requested Fourier slice k (slices[s], 0 <= k < h):
 *   Uhat[s] : n1 x R complex,  sig[s] : R (descending),  Vhat[s] : n2 x R complex
 *   err2[s] : || Xhat_k - Uhat diag(sig) Vhat^H ||_F^2
 *   m_used[s]: number of basis columns actually used (m_eff)
 * Omega: real (n3, n2, R+P) spatial test tensor, or NULL to draw it with
 * orc_gaussian(seed, 0, 0, .).  mode selects Alg. 2 (canonical or literal),
 * Alg. 1, or the exact truncated T-SVD (Omega, P, q ignored).
 */
int orc_rtsvd_fourier(const double* X, int n1, int n2, int n3, int R, int P, int q, int mode,
                      const double* Omega, uint64_t seed, const int* slices, int ns,
                      orc_cplx* Uhat, double* sig, orc_cplx* Vhat, double* err2, int* m_used);
/* The orthonormal range basis Q of the chosen mode for the requested slices:
 * Qhat[s] is n1 x m (m = returned value, the same for every slice). */
int orc_range_basis_fourier(const double* X, int n1, int n2, int n3, int R, int P, int q, int mode,
                            const double* Omega, uint64_t seed, const int* slices, int ns, orc_cplx* Qhat);
/* the same on Fourier slices given directly: Xhat (ns,n1,n2), Omhat (ns,n2,R+P) */
int orc_rtsvd_hat(const orc_cplx* Xhat, const orc_cplx* Omhat, int ns, int n1, int n2, int R, int P, int q, int mode,
                  orc_cplx* Uhat, double* sig, orc_cplx* Vhat, double* err2, int* m_used);
/* spatial factors U (n3,n1,R), S tubes (n3,R), V (n3,n2,R) from all h Fourier slices */
int orc_rtsvd(const double* X, int n1, int n2, int n3, int R, int P, int q, int mode,
              const double* Omega, uint64_t seed, double* U, double* S, double* V, double* sig_hat);
/* X_R = U * S * V^T from spatial factors (S given as (n3,R) f-diagonal tubes) */
int orc_reconstruct(const double* U, const double* S, const double* V, int n1, int n2, int n3, int R, double* Xr);

/* Alg. TQR: X (n3,n1,n2) = Q * R with Q (n3,n1,p), R (n3,p,n2), p = min(n1,n2);
 * per Fourier slice the economy QR with the diagonal of R real and >= 0. */
int orc_tqr(const double* X, int n1, int n2, int n3, double* Q, double* R);
/* Alg. mp: Moore-Penrose pseudoinverse Xp (n3,n2,n1) of X (n3,n1,n2). */
int orc_tpinv(const double* X, int n1, int n2, int n3, double* Xp);
/* Ex. 3: C <- T ? M : X element-wise, returns sum (C_new - C_old)^2; and the PSNR (Sec. 5) */
double orc_fill_in(double* C, const double* M, const unsigned char* T, const double* X, long n);
double orc_psnr(const double* X, const double* Y, long n, double peak);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
