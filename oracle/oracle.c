/*
 * oracle.c -- plain FP64 CPU oracle for the randomized block Krylov truncated
 * T-SVD (Kooshkghazi, Ahmadi-Asl, de Almeida, arXiv 2504.04989).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * cpu_baseline leg of bench.py, never by the product path.  It is written for
 * a reader checking it against the paper: naive loops, FP64 throughout, no
 * BLAS/LAPACK/FFT library, OpenMP only across independent Fourier slices.
 *
 * Parity pins live in tests/test_oracle.py; every function below names the
 * passage it follows.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef orc_cplx cplx;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ========================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as     */
/* easy as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies with the    */
/* published multipliers and Weyl key increments.                              */
/* ========================================================================== */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Reading of randn (Alg. 1 and Alg. 2, first line): element e of a stream is
 * drawn from Philox call e/4 with counter (e/4 low word, e/4 high word, stream,
 * tensor id) and key (seed low, seed high).  Words (x0,x1) and (x2,x3) each give
 * two normals by Box-Muller with uniforms u = (x + 1) 2^-32 in (0, 1]. */
void orc_gaussian(uint64_t seed, uint32_t stream, uint32_t tensor_id, long n, double* out) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two32inv = 1.0 / 4294967296.0;
#pragma omp parallel for schedule(static)
  for (long call = 0; call < (n + 3) / 4; ++call) {
    uint32_t ctr[4] = {(uint32_t)call, (uint32_t)((uint64_t)call >> 32), stream, tensor_id};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double z[4];
    for (int pair = 0; pair < 2; ++pair) {
      double u1 = ((double)x[2 * pair] + 1.0) * two32inv;
      double u2 = ((double)x[2 * pair + 1] + 1.0) * two32inv;
      double r = sqrt(-2.0 * log(u1));
      double theta = 2.0 * M_PI * u2;
      z[2 * pair] = r * cos(theta);
      z[2 * pair + 1] = r * sin(theta);
    }
    for (int s = 0; s < 4; ++s) {
      long e = 4 * call + s;
      if (e < n) out[e] = z[s];
    }
  }
}

/* ========================================================================== */
/* DFT along mode 3 (Sec. 2, Definition of F_n: omega = exp(-2 pi i / n),      */
/* unnormalised forward transform, F^{-1} = F^* / n).                          */
/* ========================================================================== */
static cplx omega_pow(long p, int n, int sign) {
  long r = p % n;
  if (r < 0) r += n;
  /* exact values on the real and imaginary axes, so the DC and Nyquist slices
   * of a real tensor come out exactly real (their T-SVD factors must be real) */
  if (r == 0) return 1.0;
  if (2 * r == n) return -1.0;
  if (4 * r == n) return (sign > 0) ? I : -I;
  if (4 * r == 3 * (long)n) return (sign > 0) ? -I : I;
  double ang = (double)sign * 2.0 * M_PI * (double)r / (double)n;
  return cos(ang) + I * sin(ang);
}

int orc_dft_mode3(const double* X, int n1, int n2, int n3, const int* slices, int ns, cplx* Xhat) {
  if (n1 < 1 || n2 < 1 || n3 < 1) return -1;
  const int h = n3 / 2 + 1;
  if (!slices) ns = h;
  for (int s = 0; s < ns; ++s) {
    int k = slices ? slices[s] : s;
    if (k < 0 || k >= h) return -1;
  }
  const long plane = (long)n1 * n2;
  for (int s = 0; s < ns; ++s) {
    const int k = slices ? slices[s] : s;
    cplx* w = (cplx*)malloc(sizeof(cplx) * n3);
    for (int t = 0; t < n3; ++t) w[t] = omega_pow((long)k * t, n3, -1);
#pragma omp parallel for schedule(static)
    for (long e = 0; e < plane; ++e) {
      cplx acc = 0;
      for (int t = 0; t < n3; ++t) acc += X[(long)t * plane + e] * w[t];
      Xhat[(long)s * plane + e] = acc;
    }
    free(w);
  }
  return 0;
}

/* Alg. TP (mirror loop): slices h..n3-1 of the full spectrum are the conjugates
 * of slices n3-k; then the inverse DFT x_t = (1/n3) sum_k Xbar_k omega^{-kt}. */
int orc_idft_mode3(const cplx* Xhat, int n1, int n2, int n3, double* X) {
  if (n1 < 1 || n2 < 1 || n3 < 1) return -1;
  const int h = n3 / 2 + 1;
  const long plane = (long)n1 * n2;
#pragma omp parallel for schedule(static)
  for (long e = 0; e < plane; ++e) {
    for (int t = 0; t < n3; ++t) {
      cplx acc = 0;
      for (int k = 0; k < n3; ++k) {
        cplx xk = (k < h) ? Xhat[(long)k * plane + e] : conj(Xhat[(long)(n3 - k) * plane + e]);
        acc += xk * omega_pow((long)k * t, n3, +1);
      }
      X[(long)t * plane + e] = creal(acc) / (double)n3;
    }
  }
  return 0;
}

/* ========================================================================== */
/* Dense complex helpers (row-major).                                          */
/* ========================================================================== */
/* C (M x N) = op(A) op(B); op 'N' = as stored, 'H' = conjugate transpose.
 * A is M x K ('N') or K x M ('H'); B is K x N ('N') or N x K ('H'). */
static void cgemm(char opA, char opB, int M, int N, int K, const cplx* A, const cplx* B, cplx* C) {
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      cplx acc = 0;
      for (int l = 0; l < K; ++l) {
        cplx a = (opA == 'N') ? A[(long)i * K + l] : conj(A[(long)l * M + i]);
        cplx b = (opB == 'N') ? B[(long)l * N + j] : conj(B[(long)j * K + l]);
        acc += a * b;
      }
      C[(long)i * N + j] = acc;
    }
}

/* copy columns [c0, c0+nc) of an M x ld matrix into an M x nc matrix */
static void take_cols(int M, int ld, const cplx* A, int c0, int nc, cplx* out) {
  for (int i = 0; i < M; ++i)
    for (int c = 0; c < nc; ++c) out[(long)i * nc + c] = A[(long)i * ld + c0 + c];
}

static void put_cols(int M, int ld, cplx* A, int c0, int nc, const cplx* in) {
  for (int i = 0; i < M; ++i)
    for (int c = 0; c < nc; ++c) A[(long)i * ld + c0 + c] = in[(long)i * nc + c];
}

/* ========================================================================== */
/* Economy Householder QR (the per-slice qr(.,0) of Alg. TQR).                 */
/* Column j: x = A(j:,j), alpha = -e^{i arg x_0} ||x||, v = x - alpha e_1      */
/* normalised, H_j = I - 2 v v^H.  Q = H_0 ... H_{N-1} [I_N; 0].  A zero column */
/* gives H_j = I, so Q always has orthonormal columns.                         */
/* ========================================================================== */
int orc_householder_qr(int M, int N, const cplx* X, cplx* Q, cplx* Rf) {
  if (M < 1 || N < 1 || M < N) return -1;
  cplx* A = (cplx*)malloc(sizeof(cplx) * (long)M * N);
  cplx* V = (cplx*)calloc((long)M * N, sizeof(cplx)); /* column j holds v_j (rows j..M-1) */
  memcpy(A, X, sizeof(cplx) * (long)M * N);
  for (int j = 0; j < N; ++j) {
    double nrm2 = 0;
    for (int i = j; i < M; ++i) nrm2 += creal(A[(long)i * N + j] * conj(A[(long)i * N + j]));
    double nrm = sqrt(nrm2);
    if (nrm == 0.0) continue; /* H_j = I */
    cplx x0 = A[(long)j * N + j];
    cplx phase = (cabs(x0) > 0) ? x0 / cabs(x0) : 1.0;
    cplx alpha = -phase * nrm;
    double vn2 = 0;
    for (int i = j; i < M; ++i) {
      cplx vi = A[(long)i * N + j] - ((i == j) ? alpha : 0);
      V[(long)i * N + j] = vi;
      vn2 += creal(vi * conj(vi));
    }
    double vn = sqrt(vn2);
    for (int i = j; i < M; ++i) V[(long)i * N + j] /= vn;
    for (int c = j; c < N; ++c) { /* A(j:, c) -= 2 v (v^H A(j:, c)) */
      cplx d = 0;
      for (int i = j; i < M; ++i) d += conj(V[(long)i * N + j]) * A[(long)i * N + c];
      for (int i = j; i < M; ++i) A[(long)i * N + c] -= 2.0 * V[(long)i * N + j] * d;
    }
  }
  if (Rf)
    for (int i = 0; i < N; ++i)
      for (int c = 0; c < N; ++c) Rf[(long)i * N + c] = (c >= i) ? A[(long)i * N + c] : 0;
  /* Q = H_0 ... H_{N-1} E with E = first N columns of I_M */
  for (int i = 0; i < M; ++i)
    for (int c = 0; c < N; ++c) Q[(long)i * N + c] = (i == c) ? 1.0 : 0.0;
  for (int j = N - 1; j >= 0; --j) {
    for (int c = 0; c < N; ++c) {
      cplx d = 0;
      for (int i = j; i < M; ++i) d += conj(V[(long)i * N + j]) * Q[(long)i * N + c];
      for (int i = j; i < M; ++i) Q[(long)i * N + c] -= 2.0 * V[(long)i * N + j] * d;
    }
  }
  free(A);
  free(V);
  return 0;
}

/* ========================================================================== */
/* One-sided (Hestenes) Jacobi SVD, used for the per-slice SVD of T-SVD (Sec. 2)*/
/* Columns a_p, a_q with alpha=|a_p|^2, beta=|a_q|^2, gamma=a_p^H a_q are made  */
/* orthogonal by [a_p, a_q] <- [c a_p - s e^{-i phi} a_q, s a_p + c e^{-i phi} a_q]*/
/* with phi = arg gamma, zeta = (beta-alpha)/(2|gamma|),                        */
/* t = sign(zeta)/(|zeta| + sqrt(1+zeta^2)), c = 1/sqrt(1+t^2), s = c t.        */
/* The same rotations accumulate V; X = W diag(s) V^H at convergence.           */
/* ========================================================================== */
int orc_jacobi_svd(int M, int N, const cplx* X, cplx* W, double* s, cplx* V) {
  if (M < 1 || N < 1 || M < N) return -1;
  cplx* a = (cplx*)malloc(sizeof(cplx) * (long)N * M); /* a[c*M + i] = X(i, c): columns contiguous */
  cplx* v = (cplx*)calloc((long)N * N, sizeof(cplx));  /* v[c*N + r] = V(r, c) */
  for (int i = 0; i < M; ++i)
    for (int c = 0; c < N; ++c) a[(long)c * M + i] = X[(long)i * N + c];
  for (int c = 0; c < N; ++c) v[(long)c * N + c] = 1.0;
  const double tol = sqrt((double)M) * DBL_EPSILON;
  const int max_sweeps = 80;
  int sweep = 0, converged = 0;
  while (!converged && sweep < max_sweeps) {
    ++sweep;
    converged = 1;
    for (int p = 0; p < N - 1; ++p)
      for (int q = p + 1; q < N; ++q) {
        cplx* ap = a + (long)p * M;
        cplx* aq = a + (long)q * M;
        double alpha = 0, beta = 0;
        cplx gamma = 0;
        for (int i = 0; i < M; ++i) {
          alpha += creal(ap[i] * conj(ap[i]));
          beta += creal(aq[i] * conj(aq[i]));
          gamma += conj(ap[i]) * aq[i];
        }
        double g = cabs(gamma);
        if (alpha == 0.0 || beta == 0.0 || g <= tol * sqrt(alpha) * sqrt(beta)) continue;
        converged = 0;
        cplx ephi_conj = conj(gamma) / g; /* e^{-i phi} */
        double zeta = (beta - alpha) / (2.0 * g);
        double t = ((zeta >= 0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < M; ++i) {
          cplx x = ap[i], y = aq[i] * ephi_conj;
          ap[i] = c * x - sn * y;
          aq[i] = sn * x + c * y;
        }
        cplx* vp = v + (long)p * N;
        cplx* vq = v + (long)q * N;
        for (int r = 0; r < N; ++r) {
          cplx x = vp[r], y = vq[r] * ephi_conj;
          vp[r] = c * x - sn * y;
          vq[r] = sn * x + c * y;
        }
      }
  }
  /* singular values are the column norms; order descending, ties by index */
  double* nrm = (double*)malloc(sizeof(double) * N);
  int* order = (int*)malloc(sizeof(int) * N);
  for (int c = 0; c < N; ++c) {
    double s2 = 0;
    for (int i = 0; i < M; ++i) s2 += creal(a[(long)c * M + i] * conj(a[(long)c * M + i]));
    nrm[c] = sqrt(s2);
    order[c] = c;
  }
  for (int i = 1; i < N; ++i) { /* insertion sort: stable */
    int key = order[i], j = i - 1;
    while (j >= 0 && nrm[order[j]] < nrm[key]) { order[j + 1] = order[j]; --j; }
    order[j + 1] = key;
  }
  for (int k = 0; k < N; ++k) {
    int c = order[k];
    s[k] = nrm[c];
    for (int i = 0; i < M; ++i) W[(long)i * N + k] = (nrm[c] > 0) ? a[(long)c * M + i] / nrm[c] : 0;
    for (int r = 0; r < N; ++r) V[(long)r * N + k] = v[(long)c * N + r];
  }
  free(a); free(v); free(nrm); free(order);
  return converged ? sweep : -2;
}

/* ========================================================================== */
/* t-algebra in the spatial domain (Sec. 2).                                   */
/* ========================================================================== */
/* Alg. TP: DFT both factors, multiply the h non-redundant slices, mirror, iDFT */
int orc_tprod(const double* A, const double* B, int n1, int n2, int n4, int n3, double* C) {
  if (n1 < 1 || n2 < 1 || n4 < 1 || n3 < 1) return -1;
  const int h = n3 / 2 + 1;
  cplx* Ah = (cplx*)malloc(sizeof(cplx) * (long)h * n1 * n2);
  cplx* Bh = (cplx*)malloc(sizeof(cplx) * (long)h * n2 * n4);
  cplx* Ch = (cplx*)malloc(sizeof(cplx) * (long)h * n1 * n4);
  orc_dft_mode3(A, n1, n2, n3, NULL, 0, Ah);
  orc_dft_mode3(B, n2, n4, n3, NULL, 0, Bh);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < h; ++k)
    cgemm('N', 'N', n1, n4, n2, Ah + (long)k * n1 * n2, Bh + (long)k * n2 * n4, Ch + (long)k * n1 * n4);
  orc_idft_mode3(Ch, n1, n4, n3, C);
  free(Ah); free(Bh); free(Ch);
  return 0;
}

/* Definition of the t-product: fold(bcirc(A) unfold(B)).  Block (r, c) of
 * bcirc(A) is the frontal slice A^{((r - c) mod n3)} (0-based), so
 * C^{(r)} = sum_c A^{((r-c) mod n3)} B^{(c)}.  No transform is involved. */
int orc_tprod_bcirc(const double* A, const double* B, int n1, int n2, int n4, int n3, double* C) {
  if (n1 < 1 || n2 < 1 || n4 < 1 || n3 < 1) return -1;
  memset(C, 0, sizeof(double) * (long)n3 * n1 * n4);
  for (int r = 0; r < n3; ++r)
    for (int c = 0; c < n3; ++c) {
      const double* As = A + (long)(((r - c) % n3 + n3) % n3) * n1 * n2;
      const double* Bs = B + (long)c * n2 * n4;
      double* Cs = C + (long)r * n1 * n4;
      for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n4; ++j) {
          double acc = 0;
          for (int l = 0; l < n2; ++l) acc += As[(long)i * n2 + l] * Bs[(long)l * n4 + j];
          Cs[(long)i * n4 + j] += acc;
        }
    }
  return 0;
}

/* Definition of the tensor transpose: transpose every frontal slice, and
 * reverse the order of slices 2..n3 (1-based): AT(:,:,0) = A(:,:,0)^T,
 * AT(:,:,k) = A(:,:,n3-k)^T for k >= 1 (0-based). */
int orc_ttranspose(const double* A, int n1, int n2, int n3, double* AT) {
  if (n1 < 1 || n2 < 1 || n3 < 1) return -1;
  for (int k = 0; k < n3; ++k) {
    int src = (k == 0) ? 0 : n3 - k;
    for (int i = 0; i < n2; ++i)
      for (int j = 0; j < n1; ++j) AT[(long)k * n1 * n2 + (long)i * n1 + j] = A[(long)src * n1 * n2 + (long)j * n2 + i];
  }
  return 0;
}

/* Gradient of L = <dC, A*B> (inner product of Sec. 2).  bcirc(X^T) = bcirc(X)^T
 * (Lemma on bcirc) makes the adjoint of the t-product the t-product with the
 * transpose: dA = dC * B^T, dB = A^T * dC. */
int orc_tprod_backward(const double* A, const double* B, const double* dC, int n1, int n2, int n4, int n3,
                       double* dA, double* dB) {
  if (n1 < 1 || n2 < 1 || n4 < 1 || n3 < 1) return -1;
  double* BT = (double*)malloc(sizeof(double) * (long)n3 * n4 * n2);
  double* AT = (double*)malloc(sizeof(double) * (long)n3 * n2 * n1);
  orc_ttranspose(B, n2, n4, n3, BT);
  orc_ttranspose(A, n1, n2, n3, AT);
  orc_tprod(dC, BT, n1, n4, n2, n3, dA);
  orc_tprod(AT, dC, n2, n1, n4, n3, dB);
  free(BT); free(AT);
  return 0;
}

/* Gradient of L = <dY, Q*Q^T*A> (the projection Q*Q^T*A of Sec. 4):
 * dA = Q*(Q^T*dY),  dQ = dY*(A^T*Q) + A*(dY^T*Q).  Q: n1 x m, A, dY: n1 x n2. */
int orc_tproj_backward(const double* Q, const double* A, const double* dY, int n1, int m, int n2, int n3,
                       double* dQ, double* dA) {
  if (n1 < 1 || m < 1 || n2 < 1 || n3 < 1) return -1;
  double* QT = (double*)malloc(sizeof(double) * (long)n3 * m * n1);
  double* AT = (double*)malloc(sizeof(double) * (long)n3 * n2 * n1);
  double* dYT = (double*)malloc(sizeof(double) * (long)n3 * n2 * n1);
  double* QTdY = (double*)malloc(sizeof(double) * (long)n3 * m * n2);
  double* ATQ = (double*)malloc(sizeof(double) * (long)n3 * n2 * m);
  double* dYTQ = (double*)malloc(sizeof(double) * (long)n3 * n2 * m);
  double* tmp = (double*)malloc(sizeof(double) * (long)n3 * n1 * m);
  orc_ttranspose(Q, n1, m, n3, QT);
  orc_ttranspose(A, n1, n2, n3, AT);
  orc_ttranspose(dY, n1, n2, n3, dYT);
  orc_tprod(QT, dY, m, n1, n2, n3, QTdY);
  orc_tprod(Q, QTdY, n1, m, n2, n3, dA);
  orc_tprod(AT, Q, n2, n1, m, n3, ATQ);
  orc_tprod(dY, ATQ, n1, n2, m, n3, dQ);
  orc_tprod(dYT, Q, n2, n1, m, n3, dYTQ);
  orc_tprod(A, dYTQ, n1, n2, m, n3, tmp);
  for (long e = 0; e < (long)n3 * n1 * m; ++e) dQ[e] += tmp[e];
  free(QT); free(AT); free(dYT); free(QTdY); free(ATQ); free(dYTQ); free(tmp);
  return 0;
}

/* ========================================================================== */
/* Randomized truncated T-SVD, one Fourier slice (Sec. 3 and the remark at the */
/* start of Sec. 4 that the method acts on each Fourier slice independently).  */
/* ========================================================================== */

/* Append the orthonormal basis of W (n1 x nb) to Qb (n1 x ldq, first c columns
 * filled): two classical Gram-Schmidt passes W <- W - Q (Q^H W), then the Q
 * factor of a Householder QR of [Q, W]; its trailing nb columns are the new
 * block (orthonormal to Q even when W is rank deficient). */
static void append_orth(int n1, int ldq, cplx* Qb, int c, const cplx* W0, int nb) {
  cplx* W = (cplx*)malloc(sizeof(cplx) * (long)n1 * nb);
  memcpy(W, W0, sizeof(cplx) * (long)n1 * nb);
  if (c > 0) {
    cplx* Q = (cplx*)malloc(sizeof(cplx) * (long)n1 * c);
    cplx* P = (cplx*)malloc(sizeof(cplx) * (long)c * nb);
    cplx* QP = (cplx*)malloc(sizeof(cplx) * (long)n1 * nb);
    take_cols(n1, ldq, Qb, 0, c, Q);
    for (int pass = 0; pass < 2; ++pass) {
      cgemm('H', 'N', c, nb, n1, Q, W, P);
      cgemm('N', 'N', n1, nb, c, Q, P, QP);
      for (long e = 0; e < (long)n1 * nb; ++e) W[e] -= QP[e];
    }
    free(Q); free(P); free(QP);
  }
  const int nc = c + nb;
  cplx* M = (cplx*)malloc(sizeof(cplx) * (long)n1 * nc);
  cplx* Qh = (cplx*)malloc(sizeof(cplx) * (long)n1 * nc);
  for (int i = 0; i < n1; ++i) {
    for (int j = 0; j < c; ++j) M[(long)i * nc + j] = Qb[(long)i * ldq + j];
    for (int j = 0; j < nb; ++j) M[(long)i * nc + c + j] = W[(long)i * nb + j];
  }
  orc_householder_qr(n1, nc, M, Qh, NULL);
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < nb; ++j) Qb[(long)i * ldq + c + j] = Qh[(long)i * nc + c + j];
  free(M); free(Qh); free(W);
}

/* plain orth(W): Q factor of the Householder QR (Alg. TQR per slice) */
static void orth(int n1, int nb, const cplx* W, cplx* Q) { orc_householder_qr(n1, nb, W, Q, NULL); }

/* Basis Q (n1 x m, returned m) of the range sketch of Xk for the chosen mode.
 *   ORC_ALG2_CANONICAL: Q_0 = orth(Xk Om); for i = 1..q,
 *       W_i = Xk (Xk^H Q_{i-1}), Q_i = W_i orthonormalised against Q_0..Q_{i-1};
 *       same span as T-QR of K = [K_0, ..., K_q] (Alg. 2) in exact arithmetic.
 *   ORC_ALG2_LITERAL: K_0 = Xk Om, K_i = Xk Xk^H K_{i-1}, Q = Householder Q of
 *       the first m columns of [K_0, ..., K_q] (Alg. 2 as printed).
 *   ORC_ALG1_POWER: Q = orth(Y_q) with Y_0 = Xk Om, Y_i = Xk Xk^H Y_{i-1}
 *       (Alg. 1), orthonormalising after every step (same span).
 * m = min((q+1) b, n1, n2) for Alg. 2 and min(b, n1, n2) for Alg. 1; the last
 * block keeps its leading columns only. */
static int range_basis(const cplx* Xk, const cplx* Om, int n1, int n2, int b, int q, int mode, cplx* Qb) {
  const int mtot = (mode == ORC_ALG1_POWER) ? b : (q + 1) * b;
  int m = mtot;
  if (m > n1) m = n1;
  if (m > n2) m = n2;
  const int b0 = (b < m) ? b : m;
  cplx* W = (cplx*)malloc(sizeof(cplx) * (long)n1 * b);
  cplx* Y = (cplx*)malloc(sizeof(cplx) * (long)n2 * b);
  cplx* Qprev = (cplx*)malloc(sizeof(cplx) * (long)n1 * b);
  cplx* Omb = (cplx*)malloc(sizeof(cplx) * (long)n2 * b0);
  take_cols(n2, b, Om, 0, b0, Omb);
  cgemm('N', 'N', n1, b0, n2, Xk, Omb, W); /* K_0 = X * B */
  if (mode == ORC_ALG2_CANONICAL) {
    append_orth(n1, m, Qb, 0, W, b0);
    int c = b0, pw = b0;
    for (int i = 1; i <= q && c < m; ++i) {
      const int bi = (b < m - c) ? b : m - c;
      take_cols(n1, m, Qb, c - pw, pw, Qprev);
      cgemm('H', 'N', n2, pw, n1, Xk, Qprev, Y); /* Y = Xk^H Q_{i-1} */
      cplx* Yb = (cplx*)malloc(sizeof(cplx) * (long)n2 * bi);
      take_cols(n2, pw, Y, 0, bi, Yb);
      cgemm('N', 'N', n1, bi, n2, Xk, Yb, W); /* leading columns of Xk Xk^H Q_{i-1} */
      free(Yb);
      append_orth(n1, m, Qb, c, W, bi);
      c += bi;
      pw = bi;
    }
  } else if (mode == ORC_ALG2_LITERAL) {
    cplx* K = (cplx*)malloc(sizeof(cplx) * (long)n1 * m);
    put_cols(n1, m, K, 0, b0, W);
    int c = b0, pw = b0;
    cplx* Kprev = (cplx*)malloc(sizeof(cplx) * (long)n1 * b);
    memcpy(Kprev, W, sizeof(cplx) * (long)n1 * b0);
    for (int i = 1; i <= q && c < m; ++i) {
      const int bi = (b < m - c) ? b : m - c;
      cgemm('H', 'N', n2, pw, n1, Xk, Kprev, Y);
      cplx* Kn = (cplx*)malloc(sizeof(cplx) * (long)n1 * pw);
      cgemm('N', 'N', n1, pw, n2, Xk, Y, Kn); /* K_i = X * X^T * K_{i-1} */
      put_cols(n1, m, K, c, bi, Kn);          /* keeps the leading bi columns */
      memcpy(Kprev, Kn, sizeof(cplx) * (long)n1 * pw);
      free(Kn);
      c += bi;
    }
    orc_householder_qr(n1, m, K, Qb, NULL);
    free(K); free(Kprev);
  } else { /* ORC_ALG1_POWER */
    cplx* Qc = (cplx*)malloc(sizeof(cplx) * (long)n1 * b0);
    orth(n1, b0, W, Qc);
    for (int i = 1; i <= q; ++i) {
      cgemm('H', 'N', n2, b0, n1, Xk, Qc, Y);
      cgemm('N', 'N', n1, b0, n2, Xk, Y, W);
      orth(n1, b0, W, Qc);
    }
    memcpy(Qb, Qc, sizeof(cplx) * (long)n1 * b0);
    free(Qc);
  }
  free(W); free(Y); free(Qprev); free(Omb);
  return m;
}

/* One slice: basis Q, C = Q^H Xk (Alg. 2, projection), full SVD of C via the
 * Jacobi SVD of C^H (C^H = W s V^H gives C = V s W^H, so U_c = V, V_c = W),
 * then Uhat = Q U_c(:, 1:R), S_R, V_R = V_c(:, 1:R) (Alg. 2, last lines).
 * ORC_EXACT: SVD of Xk itself (T-SVD, Sec. 2) truncated to R. */
static int rtsvd_slice(const cplx* Xk, const cplx* Om, int n1, int n2, int R, int b, int q, int mode,
                       cplx* Uh, double* sg, cplx* Vh, double* err2, int* m_used) {
  int m;
  if (mode == ORC_EXACT) {
    if (n1 >= n2) {
      cplx* W = (cplx*)malloc(sizeof(cplx) * (long)n1 * n2);
      double* s = (double*)malloc(sizeof(double) * n2);
      cplx* V = (cplx*)malloc(sizeof(cplx) * (long)n2 * n2);
      orc_jacobi_svd(n1, n2, Xk, W, s, V);
      take_cols(n1, n2, W, 0, R, Uh);
      take_cols(n2, n2, V, 0, R, Vh);
      memcpy(sg, s, sizeof(double) * R);
      free(W); free(s); free(V);
    } else {
      cplx* XH = (cplx*)malloc(sizeof(cplx) * (long)n2 * n1);
      for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j) XH[(long)j * n1 + i] = conj(Xk[(long)i * n2 + j]);
      cplx* W = (cplx*)malloc(sizeof(cplx) * (long)n2 * n1);
      double* s = (double*)malloc(sizeof(double) * n1);
      cplx* V = (cplx*)malloc(sizeof(cplx) * (long)n1 * n1);
      orc_jacobi_svd(n2, n1, XH, W, s, V);
      take_cols(n1, n1, V, 0, R, Uh);
      take_cols(n2, n1, W, 0, R, Vh);
      memcpy(sg, s, sizeof(double) * R);
      free(XH); free(W); free(s); free(V);
    }
    m = (n1 < n2) ? n1 : n2;
  } else {
    int mmax = ((mode == ORC_ALG1_POWER) ? 1 : (q + 1)) * b;
    cplx* Qb = (cplx*)malloc(sizeof(cplx) * (long)n1 * mmax);
    m = range_basis(Xk, Om, n1, n2, b, q, (mode == ORC_ALG2_QTRUNC) ? ORC_ALG2_CANONICAL : mode, Qb);
    if (mode == ORC_ALG2_QTRUNC && m > b) {
      /* Ex. 1 (Sec. 5): the factor Q of Alg. 2 truncated to k + p = R + P terms
       * before the projection; read as its leading R + P columns */
      cplx* Qt = (cplx*)malloc(sizeof(cplx) * (long)n1 * b);
      take_cols(n1, m, Qb, 0, b, Qt);
      free(Qb);
      Qb = Qt;
      m = b;
    }
    cplx* CH = (cplx*)malloc(sizeof(cplx) * (long)n2 * m); /* C^H = Xk^H Q */
    cgemm('H', 'N', n2, m, n1, Xk, Qb, CH);
    cplx* W = (cplx*)malloc(sizeof(cplx) * (long)n2 * m);
    double* s = (double*)malloc(sizeof(double) * m);
    cplx* V = (cplx*)malloc(sizeof(cplx) * (long)m * m);
    orc_jacobi_svd(n2, m, CH, W, s, V);
    cplx* Uc = (cplx*)malloc(sizeof(cplx) * (long)m * R);
    take_cols(m, m, V, 0, R, Uc);
    cgemm('N', 'N', n1, R, m, Qb, Uc, Uh); /* Uhat = Q * U_c */
    take_cols(n2, m, W, 0, R, Vh);
    memcpy(sg, s, sizeof(double) * R);
    free(Qb); free(CH); free(W); free(s); free(V); free(Uc);
  }
  /* err2 = || Xk - Uh diag(sg) Vh^H ||_F^2 */
  double e2 = 0;
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j) {
      cplx acc = Xk[(long)i * n2 + j];
      for (int r = 0; r < R; ++r) acc -= Uh[(long)i * R + r] * sg[r] * conj(Vh[(long)j * R + r]);
      e2 += creal(acc * conj(acc));
    }
  *err2 = e2;
  *m_used = m;
  return 0;
}

int orc_rtsvd_fourier(const double* X, int n1, int n2, int n3, int R, int P, int q, int mode,
                      const double* Omega, uint64_t seed, const int* slices, int ns,
                      cplx* Uhat, double* sig, cplx* Vhat, double* err2, int* m_used) {
  if (n1 < 1 || n2 < 1 || n3 < 1 || R < 1 || P < 0 || q < 0) return -1;
  if (R > n1 || R > n2) return -1;
  if (mode < ORC_ALG2_CANONICAL || mode > ORC_ALG2_QTRUNC) return -1;
  const int h = n3 / 2 + 1;
  if (!slices) ns = h;
  const int b = R + P;
  cplx* Xh = (cplx*)malloc(sizeof(cplx) * (long)ns * n1 * n2);
  if (orc_dft_mode3(X, n1, n2, n3, slices, ns, Xh) != 0) { free(Xh); return -1; }
  cplx* Omh = NULL;
  if (mode != ORC_EXACT) {
    const long nom = (long)n3 * n2 * b;
    double* Om = (double*)malloc(sizeof(double) * nom);
    if (Omega) memcpy(Om, Omega, sizeof(double) * nom);
    else orc_gaussian(seed, 0, 0, nom, Om);
    Omh = (cplx*)malloc(sizeof(cplx) * (long)ns * n2 * b);
    orc_dft_mode3(Om, n2, b, n3, slices, ns, Omh);
    free(Om);
  }
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < ns; ++s) {
    rtsvd_slice(Xh + (long)s * n1 * n2, Omh ? Omh + (long)s * n2 * b : NULL, n1, n2, R, b, q, mode,
                Uhat + (long)s * n1 * R, sig + (long)s * R, Vhat + (long)s * n2 * R, err2 + s, m_used + s);
  }
  free(Xh);
  free(Omh);
  (void)h;
  return 0;
}

/* Alg. 2 (or the chosen mode) on Fourier slices given directly: Xhat (ns, n1, n2)
 * and the transformed test blocks Omhat (ns, n2, R+P); per slice as
 * orc_rtsvd_fourier (used to check the slice-sharded multi-rank path). */
int orc_rtsvd_hat(const cplx* Xhat, const cplx* Omhat, int ns, int n1, int n2, int R, int P, int q, int mode,
                  cplx* Uhat, double* sig, cplx* Vhat, double* err2, int* m_used) {
  if (ns < 1 || n1 < 1 || n2 < 1 || R < 1 || P < 0 || q < 0 || R > n1 || R > n2) return -1;
  if (mode < ORC_ALG2_CANONICAL || mode > ORC_ALG2_QTRUNC || mode == ORC_EXACT) return -1;
  const int b = R + P;
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < ns; ++s)
    rtsvd_slice(Xhat + (long)s * n1 * n2, Omhat + (long)s * n2 * b, n1, n2, R, b, q, mode, Uhat + (long)s * n1 * R,
                sig + (long)s * R, Vhat + (long)s * n2 * R, err2 + s, m_used + s);
  return 0;
}

int orc_range_basis_fourier(const double* X, int n1, int n2, int n3, int R, int P, int q, int mode,
                            const double* Omega, uint64_t seed, const int* slices, int ns, cplx* Qhat) {
  if (n1 < 1 || n2 < 1 || n3 < 1 || R < 1 || P < 0 || q < 0 || R > n1 || R > n2) return -1;
  if (mode < ORC_ALG2_CANONICAL || mode > ORC_ALG1_POWER) return -1;
  const int h = n3 / 2 + 1;
  if (!slices) ns = h;
  const int b = R + P;
  int m = ((mode == ORC_ALG1_POWER) ? 1 : (q + 1)) * b;
  if (m > n1) m = n1;
  if (m > n2) m = n2;
  cplx* Xh = (cplx*)malloc(sizeof(cplx) * (long)ns * n1 * n2);
  if (orc_dft_mode3(X, n1, n2, n3, slices, ns, Xh) != 0) { free(Xh); return -1; }
  const long nom = (long)n3 * n2 * b;
  double* Om = (double*)malloc(sizeof(double) * nom);
  if (Omega) memcpy(Om, Omega, sizeof(double) * nom);
  else orc_gaussian(seed, 0, 0, nom, Om);
  cplx* Omh = (cplx*)malloc(sizeof(cplx) * (long)ns * n2 * b);
  orc_dft_mode3(Om, n2, b, n3, slices, ns, Omh);
  free(Om);
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < ns; ++s)
    range_basis(Xh + (long)s * n1 * n2, Omh + (long)s * n2 * b, n1, n2, b, q, mode, Qhat + (long)s * n1 * m);
  free(Xh); free(Omh);
  (void)h;
  return m;
}

int orc_rtsvd(const double* X, int n1, int n2, int n3, int R, int P, int q, int mode,
              const double* Omega, uint64_t seed, double* U, double* S, double* V, double* sig_hat) {
  if (n1 < 1 || n2 < 1 || n3 < 1 || R < 1 || R > n1 || R > n2) return -1;
  const int h = n3 / 2 + 1;
  cplx* Uh = (cplx*)malloc(sizeof(cplx) * (long)h * n1 * R);
  cplx* Vh = (cplx*)malloc(sizeof(cplx) * (long)h * n2 * R);
  cplx* Sh = (cplx*)malloc(sizeof(cplx) * (long)h * R);
  double* sg = (double*)malloc(sizeof(double) * (long)h * R);
  double* e2 = (double*)malloc(sizeof(double) * h);
  int* mu = (int*)malloc(sizeof(int) * h);
  int rc = orc_rtsvd_fourier(X, n1, n2, n3, R, P, q, mode, Omega, seed, NULL, 0, Uh, sg, Vh, e2, mu);
  if (rc == 0) {
    for (long e = 0; e < (long)h * R; ++e) Sh[e] = sg[e];
    orc_idft_mode3(Uh, n1, R, n3, U);
    orc_idft_mode3(Vh, n2, R, n3, V);
    orc_idft_mode3(Sh, 1, R, n3, S);
    if (sig_hat) memcpy(sig_hat, sg, sizeof(double) * (long)h * R);
  }
  free(Uh); free(Vh); free(Sh); free(sg); free(e2); free(mu);
  return rc;
}

/* X_R = U * S * V^T with S the f-diagonal tensor whose diagonal tubes are S */
int orc_reconstruct(const double* U, const double* S, const double* V, int n1, int n2, int n3, int R, double* Xr) {
  if (n1 < 1 || n2 < 1 || n3 < 1 || R < 1) return -1;
  double* Sf = (double*)calloc((long)n3 * R * R, sizeof(double));
  for (int t = 0; t < n3; ++t)
    for (int r = 0; r < R; ++r) Sf[(long)t * R * R + (long)r * R + r] = S[(long)t * R + r];
  double* US = (double*)malloc(sizeof(double) * (long)n3 * n1 * R);
  double* VT = (double*)malloc(sizeof(double) * (long)n3 * R * n2);
  orc_tprod(U, Sf, n1, R, R, n3, US);
  orc_ttranspose(V, n2, R, n3, VT);
  orc_tprod(US, VT, n1, R, n2, n3, Xr);
  free(Sf); free(US); free(VT);
  return 0;
}

/* ========================================================================== */
/* Alg. TQR (Sec. 2): per non-redundant Fourier slice the economy QR          */
/* qr(Xbar_k, 0), the other slices by conjugate symmetry, then the inverse    */
/* DFT of both factors.  With p = min(n1, n2): Q is n1 x p x n3, R is          */
/* p x n2 x n3.  A slice wider than tall (n1 < n2) is factored on its first   */
/* n1 columns (what Householder QR of the whole slice does: the reflectors    */
/* come from those columns) and R = Q^H Xbar_k.  The QR of a slice is unique  */
/* only up to unit phases on the diagonal of R: this oracle (reading of the   */
/* paper's MATLAB qr) fixes the diagonal of R real and non-negative, which    */
/* keeps the DC and Nyquist factors real.                                     */
/* ========================================================================== */
static void qr_slice(int n1, int n2, const cplx* X, cplx* Q, cplx* R) {
  const int p = n1 < n2 ? n1 : n2;
  cplx* lead = (cplx*)malloc(sizeof(cplx) * (long)n1 * p);
  cplx* Rl = (cplx*)malloc(sizeof(cplx) * (long)p * p);
  take_cols(n1, n2, X, 0, p, lead);
  orc_householder_qr(n1, p, lead, Q, Rl);
  for (int j = 0; j < p; ++j) { /* Q <- Q D, with D = diag(phase of R_jj) */
    const cplx d = Rl[(long)j * p + j];
    const cplx ph = (cabs(d) > 0) ? d / cabs(d) : 1.0;
    for (int i = 0; i < n1; ++i) Q[(long)i * p + j] *= ph;
  }
  cgemm('H', 'N', p, n2, n1, Q, X, R); /* R = Q^H X: upper trapezoidal, real diagonal >= 0 */
  for (int i = 0; i < p; ++i) {
    for (int c = 0; c < i && c < n2; ++c) R[(long)i * n2 + c] = 0;
    R[(long)i * n2 + i] = creal(R[(long)i * n2 + i]);
  }
  free(lead);
  free(Rl);
}

int orc_tqr(const double* X, int n1, int n2, int n3, double* Q, double* R) {
  if (n1 < 1 || n2 < 1 || n3 < 1) return -1;
  const int h = n3 / 2 + 1, p = n1 < n2 ? n1 : n2;
  cplx* Xh = (cplx*)malloc(sizeof(cplx) * (long)h * n1 * n2);
  cplx* Qh = (cplx*)malloc(sizeof(cplx) * (long)h * n1 * p);
  cplx* Rh = (cplx*)malloc(sizeof(cplx) * (long)h * p * n2);
  orc_dft_mode3(X, n1, n2, n3, NULL, 0, Xh);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < h; ++k)
    qr_slice(n1, n2, Xh + (long)k * n1 * n2, Qh + (long)k * n1 * p, Rh + (long)k * p * n2);
  orc_idft_mode3(Qh, n1, p, n3, Q);
  orc_idft_mode3(Rh, p, n2, n3, R);
  free(Xh);
  free(Qh);
  free(Rh);
  return 0;
}

/* ========================================================================== */
/* Alg. mp (Sec. 2): per non-redundant Fourier slice the Moore-Penrose        */
/* pseudoinverse pinv(Xbar_k) = V diag(1/s) W^H over the singular values above */
/* the tolerance max(n1, n2) * eps * s_max (MATLAB's pinv default), from the   */
/* one-sided Jacobi SVD (of Xbar_k^H when the slice is wide, since            */
/* pinv(X) = pinv(X^H)^H); conjugate symmetry and the inverse DFT give the    */
/* n2 x n1 x n3 tensor X^dagger.                                              */
/* ========================================================================== */
static void pinv_slice(int n1, int n2, const cplx* X, cplx* Xp) {
  const int tall = n1 >= n2;
  const int M = tall ? n1 : n2, N = tall ? n2 : n1;
  cplx* A = (cplx*)malloc(sizeof(cplx) * (long)M * N);
  cplx* W = (cplx*)malloc(sizeof(cplx) * (long)M * N);
  cplx* V = (cplx*)malloc(sizeof(cplx) * (long)N * N);
  double* s = (double*)malloc(sizeof(double) * N);
  for (int i = 0; i < M; ++i)
    for (int c = 0; c < N; ++c) A[(long)i * N + c] = tall ? X[(long)i * n2 + c] : conj(X[(long)c * n2 + i]);
  orc_jacobi_svd(M, N, A, W, s, V); /* A = W diag(s) V^H */
  const double tol = (double)M * DBL_EPSILON * s[0];
  /* pinv(A) = V diag(1/s) W^H is N x M; pinv(X) = pinv(A) (tall) or pinv(A)^H (wide) */
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < M; ++c) {
      cplx acc = 0;
      for (int k = 0; k < N; ++k)
        if (s[k] > tol) acc += V[(long)r * N + k] * (1.0 / s[k]) * conj(W[(long)c * N + k]);
      if (tall) Xp[(long)r * n1 + c] = acc;   /* Xp is n2 x n1 = N x M */
      else Xp[(long)c * n1 + r] = conj(acc);  /* Xp is n2 x n1 = M x N */
    }
  free(A);
  free(W);
  free(V);
  free(s);
}

int orc_tpinv(const double* X, int n1, int n2, int n3, double* Xp) {
  if (n1 < 1 || n2 < 1 || n3 < 1) return -1;
  const int h = n3 / 2 + 1;
  cplx* Xh = (cplx*)malloc(sizeof(cplx) * (long)h * n1 * n2);
  cplx* Ph = (cplx*)malloc(sizeof(cplx) * (long)h * n2 * n1);
  orc_dft_mode3(X, n1, n2, n3, NULL, 0, Xh);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < h; ++k) pinv_slice(n1, n2, Xh + (long)k * n1 * n2, Ph + (long)k * n2 * n1);
  orc_idft_mode3(Ph, n2, n1, n3, Xp);
  free(Xh);
  free(Ph);
  return 0;
}

/* ========================================================================== */
/* Data completion, Sec. 5 Ex. 3: the fill-in C <- T .* M + (1 - T) .* X and   */
/* the squared distance behind PSNR = 10 log10(peak^2 / MSE), MSE = ||.||^2/N. */
/* ========================================================================== */
double orc_fill_in(double* C, const double* M, const unsigned char* T, const double* X, long n) {
  double change2 = 0;
  for (long i = 0; i < n; ++i) {
    const double c = T[i] ? M[i] : X[i];
    change2 += (c - C[i]) * (c - C[i]);
    C[i] = c;
  }
  return change2;
}

double orc_psnr(const double* X, const double* Y, long n, double peak) {
  double s = 0;
  for (long i = 0; i < n; ++i) s += (X[i] - Y[i]) * (X[i] - Y[i]);
  return (s == 0) ? INFINITY : 10.0 * log10(peak * peak / (s / (double)n));
}
