// tsvd_rbk.cu -- the randomized block Krylov truncated T-SVD (Alg. 2, Sec. 3)
// as one stream of kernels, and its C-ABI entry points.
//
// Per non-redundant Fourier slice k (all slices batched in every launch):
//   Omega_k          rFFT of the real Gaussian test tensor B (Alg. 2, line 1)
//   A_k              rFFT of the data tensor (Alg. TP, first line)
//   W_0 = A_k Om_k   K_0 = X * B                               (Alg. 2, line 2)
//   Q_0 = orth(W_0)
//   Y_i = A_k^H Q_{i-1},  W_i = A_k Y_i   K_i = X * X^T * K_{i-1} (Alg. 2, line 4)
//   Q_i = orth(W_i - Q_{<i} Q_{<i}^H W_i)  T-QR of K = [K_0..K_q] (Alg. 2, lines 5-6)
//   C^H = A_k^H Q = [Y_1, .., Y_q, A_k^H Q_q]  (C = Q^T * X, Alg. 2 line 7; the
//         first q blocks are the Y_i already formed by the Krylov steps)
//   G = C C^H = U_c S_c^2 U_c^H           T-SVD(C)                  (Alg. 2, line 8)
//   Uhat = Q U_c(:, 1:R),  Vhat = C^H U_c(:, 1:R) S_R^{-1}          (Alg. 2, lines 9-10)
//   inverse rFFT of Uhat, Vhat and the singular tubes.
// orth = three passes of [classical Gram-Schmidt against Q_{<i}, CholeskyQR]
// (shifted CholeskyQR3): the first Cholesky is shifted so that it cannot break
// down; columns found dependent afterwards are replaced by fresh orthonormal
// directions.  It runs in FP64 on the FP64 path and in FP32 on the FP32 path
// (FP64 on request): on GB300 FP64 arithmetic runs at 1/58 of FP32, and the
// projected Krylov blocks are well conditioned, so FP32 keeps the basis
// orthonormal to ~1e-7, far inside the path's singular-value tolerance.  The
// Gram matrix G and its eigen-solve always run in FP64.
#include <type_traits>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

struct RbkDims {
  int n1, n2, n3, h, R, P, q, b, m;
  int hfull;    // floor(n3/2) + 1 non-redundant slices of the transform
  int k0;       // first Fourier slice processed (h slices from k0 on)
  int fourier;  // the caller passes the Fourier slices (tsvd_rbk_fourier): no transforms here
  int tc;    // basis-building products on tcgen05 in one pass: 0 none, 1 TF32, 2 BF16
  int tco;   // FP32 block orthonormalisation with its Gram and W R^-1 on tcgen05 (split TF32)
  int tc3;   // FP32-accurate products on tcgen05 (split TF32): FP32 data unless TSVD_FLAG_SIMT
  int alg1;  // Alg. 1 (power iteration, last block only) instead of Alg. 2
  int gsl;   // FP32 paths: the exact Gram in its digit form on the BF16 tensor cores
  int mp;    // basis columns used by the projection: m, or R+P with TSVD_FLAG_QTRUNC
  int deflate;  // deflated Rayleigh-Ritz passes for the small SVD (FP64 path)
};

static int rbk_dims(int n1, int n2, int n3, const tsvd_params* p, RbkDims* d) {
  if (!p || n1 < 1 || n2 < 1 || n3 < 1) return TSVD_ERR_INVALID_ARG;
  if (p->R < 1 || p->P < 0 || p->q < 0 || p->R > n1 || p->R > n2) return TSVD_ERR_INVALID_ARG;
  if (p->precision < TSVD_FP64 || p->precision > TSVD_MIXED_BF16) return TSVD_ERR_INVALID_ARG;
  d->n1 = n1;
  d->n2 = n2;
  d->n3 = n3;
  d->h = n3 / 2 + 1;
  d->hfull = d->h;
  d->k0 = 0;
  d->fourier = 0;
  d->R = p->R;
  d->P = p->P;
  d->q = p->q;
  d->b = p->R + p->P;
  d->tc = (p->precision == TSVD_MIXED_TF32) ? 1 : (p->precision == TSVD_MIXED_BF16) ? 2 : 0;
  d->alg1 = (p->flags & TSVD_FLAG_ALG1) ? 1 : 0;
  d->tc3 = (p->precision != TSVD_FP64 && !(p->flags & TSVD_FLAG_SIMT)) ? 1 : 0;
  // measured: faster from n1 ~ 1024 on (2048 x 2048 x 128: 13.4 -> 7.8 ms); at n1 = 512 the SIMT
  // kernels win (0.64 -> 1.18 ms), the blocks being too small to fill the tensor-core tiles
  d->tco = (d->tc3 && !(p->flags & TSVD_FLAG_FP64_QR) && n1 >= 1024) ? 1 : 0;
  if (p->flags & TSVD_FLAG_SIMT) d->tc = 0;
  long m = (long)(d->alg1 ? 1 : p->q + 1) * d->b;
  m = std::min<long>(m, std::min(n1, n2));
  d->m = (int)m;
  d->gsl = (d->tc3 && !(p->flags & TSVD_FLAG_GRAM_INT) && gram_sliced_ok(n2, d->m)) ? 1 : 0;
  d->mp = (p->flags & TSVD_FLAG_QTRUNC) ? std::min(d->b, d->m) : d->m;
  d->deflate = (p->flags & TSVD_FLAG_DEFLATE) ? 1 : 0;
  if (d->deflate && p->precision != TSVD_FP64) return TSVD_ERR_UNSUPPORTED;
  if (d->b > 128 || d->m > 512) return TSVD_ERR_UNSUPPORTED;
  if ((long)d->h * n1 * n2 > (1L << 40)) return TSVD_ERR_UNSUPPORTED;
  return TSVD_OK;
}

template <typename T>
struct RbkWs {
  using C = cx_t<T>;
  C* Ah;
  T* Om;
  C* Omh;
  void* Ql;    // basis in the orthonormalisation precision (n1 x m per slice)
  C* Qt;       // basis in the GEMM precision (alias of Ql when they agree)
  void* Wl;    // Krylov block in the orthonormalisation precision (n1 x b)
  C* Wt;       // Krylov block from the GEMMs (alias of Wl when they agree)
  void* Pl;    // Gram-Schmidt coefficients (m x b)
  void* Gl;    // block Gram matrix (b x b)
  C* CHt;
  double2* CH64;  // C^H in FP64 for the Gram (FP64 path: alias of CHt)
  int2* Qint;     // C^H as scaled integers for the exact Gram (FP32 paths; integer form)
  void* gsl;      // scratch of its digit form on the BF16 tensor cores
  int* colexp;    // their per-column exponents
  double2* Rs;
  uint32_t* dead;
  int* counters;  // [0] status, [1] dead columns
  double2* G;
  double* lam;
  C* Uct;      // U_c (m x R per slice) in the GEMM precision
  C* Uh;
  C* Vh;
  C* Sh;
  void* eig;
  void* Aop;      // one-pass BF16 operand: X-hat as real rows of 2 n2, padded
  float* Ahi;     // split TF32 operands: X-hat as real rows (leading dim lda) ...
  float* Alo;     //   (the FP32 path; the TF32 path reads X-hat itself, or a padded copy in Ahi)
  bool adirect;   // TF32 path: X-hat's own rows are the basis product's operand
  float* AThi;    // ... and X-hat^T (per slice n2 x n1 complex) as real rows (leading dim ldt)
  float* ATlo;
  long lda, ldt;
  float* Eh;      // expanded real forms of the thin factor (2b rows per slice, leading dim lde)
  float* El;
  long lde;
  int* tc_err;    // set by a tcgen05 pipeline wait that timed out
  double2* splitk;
  size_t splitk_elems;
  // deflated passes (FP64 path with TSVD_FLAG_DEFLATE)
  double* lamF;   // accepted eigenvalues (h x R)
  double2* UF;    // accepted eigenvectors (h x mp x R)
  double2* Um;    // the same, zero beyond the accepted columns
  double2* T1;    // C^H Um (h x n2 x R)
  double2* CpH;   // projected C^H (h x n2 x mp)
  int* acc;       // accepted count per slice
  OrthTc otc;     // tcgen05 operands of the FP32 block orthonormalisation (d.tco)
  size_t bytes;
};

template <typename T, typename L>
static RbkWs<T> carve_rbk(void* base, const RbkDims& d) {
  using C = cx_t<T>;
  using CL = cx_t<L>;
  constexpr bool dbl = std::is_same<T, double>::value;
  constexpr bool same = std::is_same<T, L>::value;
  Carver cv(base);
  RbkWs<T> w;
  const size_t h = d.h;
  w.Ah = d.fourier ? nullptr : cv.take<C>(h * d.n1 * d.n2);
  w.Om = cv.take<T>((size_t)d.n3 * d.n2 * d.b);
  w.Omh = cv.take<C>((size_t)d.hfull * d.n2 * d.b);
  w.Ql = cv.take<CL>(h * d.n1 * d.m);
  w.Qt = same ? (C*)w.Ql : cv.take<C>(h * d.n1 * d.m);
  w.Wl = cv.take<CL>(h * d.n1 * d.b);
  w.Wt = same ? (C*)w.Wl : cv.take<C>(h * d.n1 * d.b);
  w.Pl = cv.take<CL>(h * d.m * d.b);
  w.Gl = cv.take<CL>(h * d.b * d.b);
  w.CHt = cv.take<C>(h * d.n2 * d.m);
  w.CH64 = dbl ? (double2*)w.CHt : nullptr;
  const bool sliced = !dbl && d.gsl;
  w.Qint = (dbl || sliced) ? nullptr : cv.take<int2>(h * d.n2 * d.m);
  w.gsl = sliced ? (void*)cv.take<char>(gram_sliced_bytes(d.n2, d.m, h)) : nullptr;
  w.colexp = dbl ? nullptr : cv.take<int>(h * d.m);
  w.Rs = cv.take<double2>(h * d.b * d.b);
  w.dead = cv.take<uint32_t>(h * 4);
  w.counters = cv.take<int>(8);
  w.G = cv.take<double2>(h * d.m * d.m);
  w.lam = cv.take<double>(h * d.R);
  w.Uct = cv.take<C>(h * d.m * d.R);
  w.Uh = d.fourier ? nullptr : cv.take<C>(h * d.n1 * d.R);
  w.Vh = d.fourier ? nullptr : cv.take<C>(h * d.n2 * d.R);
  w.Sh = cv.take<C>(h * d.R);
  w.eig = cv.take<char>(eig_scratch_bytes(d.m, d.R, d.h));
  w.Aop = nullptr;
  w.Ahi = w.Alo = w.AThi = w.ATlo = w.Eh = w.El = nullptr;
  w.tc_err = nullptr;
  w.lda = (2L * d.n2 + 7) / 8 * 8;
  w.ldt = (2L * d.n1 + 7) / 8 * 8;
  w.lde = std::max(w.lda, w.ldt);
  w.adirect = false;
  if (d.tc3) {
    if (d.tc != 2) w.Ahi = cv.take<float>(h * d.n1 * w.lda);
    if (d.tc == 0) w.Alo = cv.take<float>(h * d.n1 * w.lda);
    w.AThi = cv.take<float>(h * d.n2 * w.ldt);
    w.ATlo = cv.take<float>(h * d.n2 * w.ldt);
    w.Eh = cv.take<float>(h * 2 * (size_t)d.b * w.lde);
    w.El = cv.take<float>(h * 2 * (size_t)d.b * w.lde);
    w.tc_err = cv.take<int>(4);
    if (d.tc == 2) w.Aop = cv.take<uint16_t>(h * d.n1 * w.lda);
  }
  w.otc = OrthTc{};
  if (d.tco) {
    OrthTc& t = w.otc;
    t.ldq2 = (2L * d.n1 + 7) / 8 * 8;
    t.ldw2 = (2L * d.b + 7) / 8 * 8;
    t.WThi = cv.take<float>(h * d.b * t.ldq2);
    t.WTlo = cv.take<float>(h * d.b * t.ldq2);
    t.Whi = cv.take<float>(h * d.n1 * t.ldw2);
    t.Wlo = cv.take<float>(h * d.n1 * t.ldw2);
    t.Ehi = cv.take<float>(h * 2 * (size_t)d.b * t.ldq2);
    t.Elo = cv.take<float>(h * 2 * (size_t)d.b * t.ldq2);
    t.ldqi = (2L * d.m + 7) / 8 * 8;
    t.Qhi = cv.take<float>(h * d.n1 * t.ldqi);
    t.Qlo = cv.take<float>(h * d.n1 * t.ldqi);
    t.Qdhi = cv.take<float>(h * 2 * (size_t)d.m * (t.ldq2 / 2));
    t.Qdlo = cv.take<float>(h * 2 * (size_t)d.m * (t.ldq2 / 2));
    t.err = w.tc_err;
  }
  w.splitk_elems = 8 * h * (size_t)d.m * std::max(d.b, 64);
  w.splitk = cv.take<double2>(w.splitk_elems);
  w.lamF = nullptr;
  w.UF = w.Um = w.T1 = w.CpH = nullptr;
  w.acc = nullptr;
  if (d.deflate) {
    w.lamF = cv.take<double>(h * d.R);
    w.UF = cv.take<double2>(h * d.mp * d.R);
    w.Um = cv.take<double2>(h * d.mp * d.R);
    w.T1 = cv.take<double2>(h * d.n2 * d.R);
    w.CpH = cv.take<double2>(h * d.n2 * d.mp);
    w.acc = cv.take<int>(h);
  }
  w.bytes = cv.bytes();
  return w;
}


// Orthonormalise the nb leading columns of the Krylov block W against the c
// finished columns of Q (orth_block_cols in cholqr.cu: shifted CholeskyQR3
// with classical Gram-Schmidt, dead columns replaced) in the precision L.
template <typename T, typename L>
static int orth_block(const RbkDims& d, RbkWs<T>& w, int c, int nb, int block_id, uint64_t seed, cudaStream_t s) {
  OrthWs o;
  o.Q = w.Ql;
  o.W = w.Wl;
  o.P = w.Pl;
  o.G = w.Gl;
  o.Minv = w.Rs;
  o.dead = w.dead;
  o.dead_count = w.counters + 1;
  o.Qt = std::is_same<T, L>::value ? nullptr : (void*)w.Qt;
  o.splitk = w.splitk;
  o.splitk_elems = w.splitk_elems;
  o.k0 = d.k0;
  o.nyq = (d.n3 % 2 == 0) ? d.n3 / 2 : -1;
  o.tc = d.tco ? &w.otc : nullptr;
  return orth_block_cols<L>(d.n1, d.b, d.m, d.h, o, c, nb, block_id, seed, s);
}

// Krylov block from the GEMM precision to the orthonormalisation precision
template <typename T, typename L>
static int to_orth(const RbkWs<T>& w, const RbkDims& d, int cols, cudaStream_t s) {
  if (std::is_same<T, L>::value) return TSVD_OK;
  TSVD_STAGE("convert", s);
  const long sW = (long)d.n1 * d.b;
  return convert_c32_to_c64((const float2*)w.Wt, d.b, sW, (double2*)w.Wl, d.b, sW, d.n1, cols, d.h, s);
}

// W (n1 x nb, leading dim b) = X-hat Y for the thin Y (n2 x nb, leading dim ldy):
// on tcgen05 (one TF32 / BF16 pass in the mixed precisions, split TF32 on the
// FP32 path; X-hat seen as real n1 x 2n2 rows, Y as its expanded real form),
// else the SIMT GEMM.
template <typename T>
static int basis_product(const RbkDims& d, RbkWs<T>& w, const cx_t<T>* Y, long ldy, long sy, int nb, cudaStream_t s) {
  const int n1 = d.n1, n2 = d.n2, b = d.b, h = d.h;
  const long sA = (long)n1 * n2, sW = (long)n1 * b, se = 2L * b * w.lde;
  if constexpr (std::is_same<T, float>::value) {
    if (d.tc == 2) {
      TSVD_TRY(expand_thin(Y, ldy, sy, n2, nb, w.Eh, w.lde, se, h, 0, true, s));
      return tc_gemm(w.Aop, w.lda, (long)n1 * w.lda, n1, w.Eh, w.lde, se, 2 * nb, 2 * n2, (float*)w.Wt, 2L * b,
                     2L * sW, h, true, w.tc_err, s);
    }
    if (d.tc == 1) {  // one TF32 pass on X-hat (its rows, or their padded copy)
      TSVD_TRY(expand_thin(Y, ldy, sy, n2, nb, w.Eh, w.lde, se, h, 0, false, s));
      const float* Ar = w.adirect ? (const float*)w.Ah : w.Ahi;
      const long la = w.adirect ? 2L * n2 : w.lda;
      return tc_gemm(Ar, la, (long)n1 * la, n1, w.Eh, w.lde, se, 2 * nb, 2 * n2, (float*)w.Wt, 2L * b, 2L * sW, h,
                     false, w.tc_err, s);
    }
    if (d.tc3) {
      TSVD_TRY(expand_thin_split(Y, ldy, sy, n2, nb, w.Eh, w.El, w.lde, se, h, 0, s));
      return tc_gemm_split(w.Ahi, w.Alo, w.lda, (long)n1 * w.lda, n1, w.Eh, w.El, w.lde, se, 2 * nb, 2 * n2,
                           (float*)w.Wt, 2L * b, 2L * sW, h, w.tc_err, s);
    }
  }
  return cgemm<cx_t<T>>(gemm('N', 'N', n1, nb, n2, 1.0, w.Ah, n2, sA, Y, ldy, sy, 0.0, w.Wt, b, sW, h), w.splitk,
                        w.splitk_elems * 2, s);
}

// columns [col0, col0 + nb) of C^H (n2 x m) = X-hat^H Q(:, col0 : col0 + nb): the
// products that form C, so FP32 accuracy (split TF32 on tcgen05, or SIMT)
template <typename T>
static int conj_product(const RbkDims& d, RbkWs<T>& w, int col0, int nb, cudaStream_t s) {
  const int n1 = d.n1, n2 = d.n2, m = d.m, b = d.b, h = d.h;
  const long sA = (long)n1 * n2, sQ = (long)n1 * m, sCH = (long)n2 * m, se = 2L * b * w.lde;
  if constexpr (std::is_same<T, float>::value) {
    if (d.tc3) {
      TSVD_TRY(expand_thin_split(w.Qt + col0, m, sQ, n1, nb, w.Eh, w.El, w.lde, se, h, 1, s));
      return tc_gemm_split(w.AThi, w.ATlo, w.ldt, (long)n2 * w.ldt, n2, w.Eh, w.El, w.lde, se, 2 * nb, 2 * n1,
                           (float*)(w.CHt + col0), 2L * m, 2L * sCH, h, w.tc_err, s);
    }
  }
  return cgemm<cx_t<T>>(gemm('H', 'N', n2, nb, n1, 1.0, w.Ah, n2, sA, w.Qt + col0, m, sQ, 0.0, w.CHt + col0, m, sCH,
                             h),
                        w.splitk, w.splitk_elems * 2, s);
}

// Deflated Rayleigh-Ritz passes of the small SVD (FP64 path, deflate.cu):
// pass 0 is the eigen-solve already done; each further pass projects the
// accepted directions out of C twice, re-forms the Gram and solves it.
static int deflated_passes(const RbkDims& d, RbkWs<double>& w, cudaStream_t s) {
  constexpr int kPasses = 6;  // six decades of lambda each: the whole FP64 range
  const int n2 = d.n2, m = d.m, mp = d.mp, R = d.R, h = d.h;
  const long sCH = (long)n2 * m, sU = (long)mp * R, sT = (long)n2 * R, sP = (long)n2 * mp;
  TSVD_STAGE("eig_deflate", s);
  if (cudaMemsetAsync(w.Um, 0, sizeof(double2) * (size_t)h * sU, s) != cudaSuccess) return TSVD_ERR_CUDA;
  TSVD_TRY(deflate_merge(w.lam, w.Uct, mp, R, h, w.lamF, w.UF, w.Um, w.acc, true, false, s));
  for (int pass = 1; pass < kPasses; ++pass) {
    TSVD_TRY(copy_cx<double2>(w.CH64, m, sCH, w.CpH, mp, sP, n2, mp, h, s));
    for (int sweep = 0; sweep < 2; ++sweep) {  // C_p^H <- C_p^H - (C_p^H U_m) U_m^H, twice
      TSVD_TRY(cgemm<double2>(gemm('N', 'N', n2, R, mp, 1.0, w.CpH, mp, sP, w.Um, R, sU, 0.0, w.T1, R, sT, h), w.splitk,
                              w.splitk_elems, s));
      TSVD_TRY(cgemm<double2>(gemm('N', 'H', n2, mp, R, -1.0, w.T1, R, sT, w.Um, R, sU, 1.0, w.CpH, mp, sP, h),
                              w.splitk, w.splitk_elems, s));
    }
    TSVD_TRY(cgemm_herm<double2>(gemm('H', 'N', mp, mp, n2, 1.0, w.CpH, mp, sP, w.CpH, mp, sP, 0.0, w.G, mp,
                                      (long)mp * mp, h),
                                 w.splitk, w.splitk_elems, s));
    TSVD_TRY(herm_eig_topR<double2>(w.G, mp, (long)mp * mp, mp, R, h, w.lam, w.Uct, R, sU, w.eig, w.counters, s));
    TSVD_TRY(deflate_merge(w.lam, w.Uct, mp, R, h, w.lamF, w.UF, w.Um, w.acc, false, pass == kPasses - 1, s));
  }
  if (cudaMemcpyAsync(w.lam, w.lamF, sizeof(double) * (size_t)h * R, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(w.Uct, w.UF, sizeof(double2) * (size_t)h * sU, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return TSVD_ERR_CUDA;
  return TSVD_OK;
}

template <typename T, typename L>
static int rbk_run(const T* A, const RbkDims& d, const tsvd_params& p, const T* Omega, T* U, T* S, T* V,
                   double* sig, void* ws, cudaStream_t s, tsvd_info* info, const cx_t<T>* Ahat = nullptr,
                   cx_t<T>* Uhat = nullptr, cx_t<T>* Vhat = nullptr) {
  using C = cx_t<T>;
  RbkWs<T> w = carve_rbk<T, L>(ws, d);
  if (d.fourier) {  // Fourier slices k0 .. k0+h-1 given and returned by the caller
    w.Ah = const_cast<C*>(Ahat);
    w.Uh = Uhat;
    w.Vh = Vhat;
  }
  const int n1 = d.n1, n2 = d.n2, n3 = d.n3, h = d.h, b = d.b, m = d.m, R = d.R;
  const long sQ = (long)n1 * m, sCH = (long)n2 * m, sO = (long)n2 * b;
  if (cudaMemsetAsync(w.counters, 0, 8 * sizeof(int), s) != cudaSuccess) return TSVD_ERR_CUDA;

  // test tensor and data in the Fourier domain
  const T* Om = Omega;
  if (!Om) {
    TSVD_STAGE("omega", s);
    TSVD_TRY(launch_gaussian<T>(p.seed, 0, 0, (long)n3 * n2 * b, w.Om, s));
    Om = w.Om;
  }
  {
    TSVD_STAGE("rfft", s);
    TSVD_TRY(launch_rfft3<T>(Om, w.Omh, (long)n2 * b, n3, s));
    if (!d.fourier) TSVD_TRY(launch_rfft3<T>(A, w.Ah, (long)n1 * n2, n3, s));
  }
  const C* Omh = w.Omh + (long)d.k0 * n2 * b;  // the test blocks of the slices processed here

  if (d.tc3) {  // tensor-core operands of X-hat and X-hat^T (split TF32; BF16 copy for the BF16 path)
    TSVD_STAGE("krylov_split", s);
    if (cudaMemsetAsync(w.tc_err, 0, sizeof(int), s) != cudaSuccess) return TSVD_ERR_CUDA;
    if constexpr (std::is_same<T, float>::value) {
      // the one TF32 pass of the basis products reads X-hat's FP32 rows as they are (the tensor
      // cores drop the low 13 mantissa bits) when their layout suits TMA, else a padded copy
      w.adirect = d.tc == 1 && tc_gemm_supported(w.Ah, 2L * n2, 2L * n1 * n2, w.Eh, w.lde, 2L * b * w.lde, h, false);
      if (d.tc == 0) TSVD_TRY(split_rows((const float*)w.Ah, 2L * n2, w.Ahi, w.Alo, w.lda, 2 * n2, (long)h * n1, s));
      else if (d.tc == 1 && !w.adirect)
        TSVD_TRY(copy_rows((const float*)w.Ah, 2L * n2, w.Ahi, w.lda, 2 * n2, (long)h * n1, false, s));
      TSVD_TRY(split_transpose((const float2*)w.Ah, n1, n2, h, w.AThi, w.ATlo, w.ldt, s));
      if (d.tc == 2) TSVD_TRY(copy_rows((const float*)w.Ah, 2L * n2, w.Aop, w.lda, 2 * n2, (long)h * n1, true, s));
    }
  }
  // block 0: W_0 = A Omega
  const int b0 = std::min(b, m);
  {
    TSVD_STAGE((d.tc || d.tc3) ? "krylov_gemm_tc" : "krylov_gemm", s);
    TSVD_TRY(basis_product<T>(d, w, Omh, b, sO, b0, s));
  }
  TSVD_TRY((to_orth<T, L>(w, d, b0, s)));
  TSVD_TRY((orth_block<T, L>(d, w, 0, b0, 0, p.seed, s)));
  int c = b0, pw = b0;
  if (d.alg1) {  // Alg. 1: Q <- orth(A A^H Q), q times, in place
    for (int i = 1; i <= d.q; ++i) {
      {
        TSVD_STAGE(d.tc3 ? "krylov_gemm_tc" : "krylov_gemm", s);
        TSVD_TRY(conj_product<T>(d, w, 0, b0, s));
      }
      {
        TSVD_STAGE((d.tc || d.tc3) ? "krylov_gemm_tc" : "krylov_gemm", s);
        TSVD_TRY(basis_product<T>(d, w, w.CHt, m, sCH, b0, s));
      }
      TSVD_TRY((to_orth<T, L>(w, d, b0, s)));
      TSVD_TRY((orth_block<T, L>(d, w, 0, b0, i, p.seed, s)));
    }
  }
  for (int i = 1; !d.alg1 && i <= d.q && c < m; ++i) {
    const int bi = std::min(b, m - c);
    {
    TSVD_STAGE(d.tc3 ? "krylov_gemm_tc" : "krylov_gemm", s);
    // Y_i = A^H Q_{i-1}: the block of C^H that belongs to Q_{i-1}
    TSVD_TRY(conj_product<T>(d, w, c - pw, pw, s));
    }
    {
    // W_i = A Y_i (leading bi columns)
    TSVD_STAGE((d.tc || d.tc3) ? "krylov_gemm_tc" : "krylov_gemm", s);
    TSVD_TRY(basis_product<T>(d, w, w.CHt + (c - pw), m, sCH, bi, s));
    }
    TSVD_TRY((to_orth<T, L>(w, d, bi, s)));
    TSVD_TRY((orth_block<T, L>(d, w, c, bi, i, p.seed, s)));
    c += bi;
    pw = bi;
  }
  // last block of C^H = A^H Q_last (not needed when the projection keeps only
  // the leading R+P basis columns: their block Y_1 of C^H exists already)
  if (d.mp == m || c == pw) {
  TSVD_STAGE(d.tc3 ? "krylov_gemm_tc" : "krylov_gemm", s);
  TSVD_TRY(conj_product<T>(d, w, c - pw, pw, s));
  }
  // the projection uses the leading mp columns of Q (Ex. 1's Q truncated to
  // k + p terms when mp < m) and of C^H, which C^H's leading dimension m keeps
  const int mp = d.mp;

  // G = C C^H in FP64 (FP64 path) or exactly in integers from the FP32 C^H, and its top-R eigenpairs
  {
  TSVD_STAGE("gram_c", s);
  if constexpr (std::is_same<T, double>::value) {
    TSVD_TRY(cgemm_herm<double2>(gemm('H', 'N', mp, mp, n2, 1.0, w.CH64, m, sCH, w.CH64, m, sCH, 0.0, w.G, mp,
                                      (long)mp * mp, h),
                                 w.splitk, w.splitk_elems, s));
  } else {
    if (w.gsl)
      TSVD_TRY(gram_sliced_fp32((const float2*)w.CHt, m, sCH, n2, mp, h, w.colexp, w.gsl, w.G, mp, (long)mp * mp,
                                w.tc_err, s));
    else
      TSVD_TRY(gram_int_fp32((const float2*)w.CHt, m, sCH, n2, mp, h, w.Qint, w.colexp, w.G, mp, (long)mp * mp, s));
  }
  }
  TSVD_TRY(herm_eig_topR<C>(w.G, mp, (long)mp * mp, mp, R, h, w.lam, w.Uct, R, (long)mp * R, w.eig, w.counters, s));
  if constexpr (std::is_same<T, double>::value) {
    if (d.deflate) TSVD_TRY(deflated_passes(d, w, s));
  }
  {
  TSVD_STAGE("outputs", s);
  TSVD_TRY(sigma_from_lambda<T>(w.lam, R, h, sig, w.Sh, s, w.counters));

  // Uhat = Q U_c,  Vhat = C^H U_c S^{-1}
  bool done = false;
  if constexpr (std::is_same<T, float>::value) {
    if (d.tco) {
      // split TF32 on tcgen05: Q's interleaved rows from the orthonormalisation's cache (K = 2 mp),
      // then C^H split into the same buffers (Q's are no longer needed), against E(U_c)
      const OrthTc& t = w.otc;
      const long sE = 2L * R * t.ldqi, sQi = (long)n1 * t.ldqi;
      TSVD_TRY(expand_thin_split(w.Uct, R, (long)mp * R, mp, R, t.Ehi, t.Elo, t.ldqi, sE, h, 0, s));
      TSVD_TRY(tc_gemm_split(t.Qhi, t.Qlo, t.ldqi, sQi, n1, t.Ehi, t.Elo, t.ldqi, sE, 2 * R, 2 * mp, (float*)w.Uh,
                             2L * R, 2L * n1 * R, h, w.tc_err, s));
      if (n2 <= n1) {
        TSVD_TRY(split_rows((const float*)w.CHt, 2L * m, t.Qhi, t.Qlo, t.ldqi, 2 * mp, (long)h * n2, s));
        TSVD_TRY(tc_gemm_split(t.Qhi, t.Qlo, t.ldqi, (long)n2 * t.ldqi, n2, t.Ehi, t.Elo, t.ldqi, sE, 2 * R, 2 * mp,
                               (float*)w.Vh, 2L * R, 2L * n2 * R, h, w.tc_err, s));
        done = true;
      } else {
        TSVD_TRY(cgemm<C>(gemm('N', 'N', n2, R, mp, 1.0, w.CHt, m, sCH, w.Uct, R, (long)mp * R, 0.0, w.Vh, R,
                               (long)n2 * R, h),
                          w.splitk, w.splitk_elems * 2, s));
        done = true;
      }
    }
  }
  if (!done) {
    TSVD_TRY(cgemm<C>(gemm('N', 'N', n1, R, mp, 1.0, w.Qt, m, sQ, w.Uct, R, (long)mp * R, 0.0, w.Uh, R,
                           (long)n1 * R, h),
                      w.splitk, w.splitk_elems * 2, s));
    TSVD_TRY(cgemm<C>(gemm('N', 'N', n2, R, mp, 1.0, w.CHt, m, sCH, w.Uct, R, (long)mp * R, 0.0, w.Vh, R,
                           (long)n2 * R, h),
                      w.splitk, w.splitk_elems * 2, s));
  }
  TSVD_TRY(scale_columns_inv<T>(w.Vh, R, (long)n2 * R, n2, R, w.lam, h, s));
  }
  if (!d.fourier) {
  // back to the spatial domain
  TSVD_STAGE("irfft", s);
  TSVD_TRY(launch_irfft3<T>(w.Uh, U, (long)n1 * R, n3, s));
  TSVD_TRY(launch_irfft3<T>(w.Vh, V, (long)n2 * R, n3, s));
  TSVD_TRY(launch_irfft3<T>(w.Sh, S, (long)R, n3, s));
  }

  if (info) {
    int host[8], tcerr = 0;
    if (cudaMemcpyAsync(host, w.counters, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TSVD_ERR_CUDA;
    if (w.tc_err && cudaMemcpyAsync(&tcerr, w.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return TSVD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TSVD_ERR_CUDA;
    info->status = tcerr ? TSVD_ERR_CUDA : host[0];
    info->dead_columns = host[1];
    info->m_eff = mp;
    info->reserved = 0;
  }
  return TSVD_OK;
}

}  // namespace tsvd

using namespace tsvd;

static size_t rbk_bytes(const RbkDims& d, const tsvd_params* p) {
  if (p->precision == TSVD_FP64) return carve_rbk<double, double>(nullptr, d).bytes;
  if (p->flags & TSVD_FLAG_FP64_QR) return carve_rbk<float, double>(nullptr, d).bytes;
  return carve_rbk<float, float>(nullptr, d).bytes;
}

extern "C" int tsvd_rbk_workspace_size(int n1, int n2, int n3, const tsvd_params* params, size_t* bytes) {
  if (!bytes) return TSVD_ERR_INVALID_ARG;
  RbkDims d;
  TSVD_TRY(rbk_dims(n1, n2, n3, params, &d));
  *bytes = rbk_bytes(d, params);
  return TSVD_OK;
}

extern "C" int tsvd_rbk(const void* A, int n1, int n2, int n3, const tsvd_params* params, const void* Omega, void* U,
                        void* S, void* V, double* sigma_hat, void* ws, size_t ws_bytes, void* stream,
                        tsvd_info* info) {
  RbkDims d;
  TSVD_TRY(rbk_dims(n1, n2, n3, params, &d));
  if (!A || !U || !S || !V || !ws) return TSVD_ERR_INVALID_ARG;
  if (((uintptr_t)ws & 255) != 0) return TSVD_ERR_INVALID_ARG;
  if (ws_bytes < rbk_bytes(d, params)) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (params->precision == TSVD_FP64)
    return rbk_run<double, double>((const double*)A, d, *params, (const double*)Omega, (double*)U, (double*)S,
                                   (double*)V, sigma_hat, ws, s, info);
  if (params->flags & TSVD_FLAG_FP64_QR)
    return rbk_run<float, double>((const float*)A, d, *params, (const float*)Omega, (float*)U, (float*)S, (float*)V,
                                  sigma_hat, ws, s, info);
  return rbk_run<float, float>((const float*)A, d, *params, (const float*)Omega, (float*)U, (float*)S, (float*)V,
                               sigma_hat, ws, s, info);
}

// Alg. 2 on a block of Fourier slices [k0, k0 + ns) of an n1 x n2 x n3 tensor
// whose half spectrum the caller holds (the slice-sharded multi-GPU path:
// each rank transforms its rows, an all-to-all regroups slices, each rank
// calls this on its slices).  The test tensor is drawn and transformed whole
// (as in tsvd_rbk, so every slice sees the same Omega-hat), and the outputs
// stay in the Fourier domain.
static int rbk_fourier_dims(int n1, int n2, int n3, int k0, int ns, const tsvd_params* p, RbkDims* d) {
  TSVD_TRY(rbk_dims(n1, n2, n3, p, d));
  if (k0 < 0 || ns < 1 || k0 + ns > d->hfull) return TSVD_ERR_INVALID_ARG;
  d->k0 = k0;
  d->h = ns;
  d->fourier = 1;
  return TSVD_OK;
}

extern "C" int tsvd_rbk_fourier_workspace_size(int n1, int n2, int n3, int k0, int ns, const tsvd_params* params,
                                               size_t* bytes) {
  if (!bytes) return TSVD_ERR_INVALID_ARG;
  RbkDims d;
  TSVD_TRY(rbk_fourier_dims(n1, n2, n3, k0, ns, params, &d));
  *bytes = rbk_bytes(d, params);
  return TSVD_OK;
}

extern "C" int tsvd_rbk_fourier(const void* Ahat, int n1, int n2, int n3, int k0, int ns, const tsvd_params* params,
                                const void* Omega, void* Uhat, void* Vhat, double* sigma_hat, void* ws,
                                size_t ws_bytes, void* stream, tsvd_info* info) {
  RbkDims d;
  TSVD_TRY(rbk_fourier_dims(n1, n2, n3, k0, ns, params, &d));
  if (!Ahat || !Uhat || !Vhat || !sigma_hat || !ws) return TSVD_ERR_INVALID_ARG;
  if (((uintptr_t)ws & 255) != 0) return TSVD_ERR_INVALID_ARG;
  if (ws_bytes < rbk_bytes(d, params)) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (params->precision == TSVD_FP64)
    return rbk_run<double, double>(nullptr, d, *params, (const double*)Omega, nullptr, nullptr, nullptr, sigma_hat,
                                   ws, s, info, (const double2*)Ahat, (double2*)Uhat, (double2*)Vhat);
  if (params->flags & TSVD_FLAG_FP64_QR)
    return rbk_run<float, double>(nullptr, d, *params, (const float*)Omega, nullptr, nullptr, nullptr, sigma_hat, ws,
                                  s, info, (const float2*)Ahat, (float2*)Uhat, (float2*)Vhat);
  return rbk_run<float, float>(nullptr, d, *params, (const float*)Omega, nullptr, nullptr, nullptr, sigma_hat, ws, s,
                               info, (const float2*)Ahat, (float2*)Uhat, (float2*)Vhat);
}

// ---------------------------------------------------------------------------
// Batched uneven T-SVDs (independent tensors of different shapes and ranks):
// a host-side scheduler over a pool of CUDA streams.  Tensors are ordered by
// an estimate of their work (largest first) and each goes to the lane with
// the least work so far; a lane runs its tensors one after another in its
// own region of the workspace (the largest its tensors need), lanes run
// concurrently.  The lanes fork from and join back to the caller's stream
// through events, so the whole batch can be captured into one CUDA graph.
// ---------------------------------------------------------------------------
namespace tsvd {

constexpr int kMaxLanes = 32;
constexpr int kMaxDevicesBatched = 64;

struct LanePool {
  cudaStream_t s[kMaxLanes];
  cudaEvent_t done[kMaxLanes];
  cudaEvent_t fork;
  bool ready;
};
static LanePool g_lanes[kMaxDevicesBatched];
static std::mutex g_lanes_mu;

static int lane_pool(LanePool** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesBatched) return TSVD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_lanes_mu);
  LanePool& lp = g_lanes[dev];
  if (!lp.ready) {
    for (int l = 0; l < kMaxLanes; ++l) {
      if (cudaStreamCreateWithFlags(&lp.s[l], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&lp.done[l], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return TSVD_ERR_CUDA;
      }
    }
    if (cudaEventCreateWithFlags(&lp.fork, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    lp.ready = true;
  }
  *out = &lp;
  return TSVD_OK;
}

// work estimate of one T-SVD: Krylov products, orthonormalisation, eigen-solve
static double rbk_cost(const RbkDims& d) {
  const double n1 = d.n1, n2 = d.n2, m = d.m;
  return d.h * (8.0 * n1 * n2 * 2.0 * m + 16.0 * n1 * m * m + (16.0 / 3.0) * m * m * m) + 2e6;
}

struct BatchPlan {
  std::vector<int> order;    // tensors, largest first
  std::vector<int> lane_of;  // lane of each tensor
  size_t lane_off[kMaxLanes + 1];
  int lanes;
};

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

static int plan_batch(const tsvd_rbk_desc* descs, int count, int lanes, BatchPlan* bp) {
  if (!descs || count < 0 || lanes < 1) return TSVD_ERR_INVALID_ARG;
  bp->lanes = std::max(1, std::min({lanes, kMaxLanes, std::max(count, 1)}));
  std::vector<double> cost(count);
  std::vector<size_t> bytes(count);
  for (int i = 0; i < count; ++i) {
    RbkDims d;
    TSVD_TRY(rbk_dims(descs[i].n1, descs[i].n2, descs[i].n3, &descs[i].params, &d));
    cost[i] = rbk_cost(d);
    bytes[i] = align256(rbk_bytes(d, &descs[i].params));
  }
  bp->order.resize(count);
  for (int i = 0; i < count; ++i) bp->order[i] = i;
  std::stable_sort(bp->order.begin(), bp->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  bp->lane_of.assign(count, 0);
  double load[kMaxLanes] = {0};
  size_t lane_bytes[kMaxLanes] = {0};
  for (int i : bp->order) {
    int best = 0;
    for (int l = 1; l < bp->lanes; ++l)
      if (load[l] < load[best]) best = l;
    bp->lane_of[i] = best;
    load[best] += cost[i];
    lane_bytes[best] = std::max(lane_bytes[best], bytes[i]);
  }
  bp->lane_off[0] = 0;
  for (int l = 0; l < bp->lanes; ++l) bp->lane_off[l + 1] = bp->lane_off[l] + lane_bytes[l];
  return TSVD_OK;
}

static int rbk_one(const tsvd_rbk_desc& t, void* ws, cudaStream_t s) {
  RbkDims d;
  TSVD_TRY(rbk_dims(t.n1, t.n2, t.n3, &t.params, &d));
  if (!t.A || !t.U || !t.S || !t.V) return TSVD_ERR_INVALID_ARG;
  const tsvd_params& p = t.params;
  if (p.precision == TSVD_FP64)
    return rbk_run<double, double>((const double*)t.A, d, p, (const double*)t.Omega, (double*)t.U, (double*)t.S,
                                   (double*)t.V, t.sigma_hat, ws, s, nullptr);
  if (p.flags & TSVD_FLAG_FP64_QR)
    return rbk_run<float, double>((const float*)t.A, d, p, (const float*)t.Omega, (float*)t.U, (float*)t.S,
                                  (float*)t.V, t.sigma_hat, ws, s, nullptr);
  return rbk_run<float, float>((const float*)t.A, d, p, (const float*)t.Omega, (float*)t.U, (float*)t.S, (float*)t.V,
                               t.sigma_hat, ws, s, nullptr);
}

}  // namespace tsvd

extern "C" int tsvd_rbk_batched_workspace_size(const tsvd_rbk_desc* descs, int count, int lanes, size_t* bytes) {
  if (!bytes) return TSVD_ERR_INVALID_ARG;
  BatchPlan bp;
  TSVD_TRY(plan_batch(descs, count, lanes, &bp));
  *bytes = bp.lane_off[bp.lanes];
  return TSVD_OK;
}

extern "C" int tsvd_rbk_batched(const tsvd_rbk_desc* descs, int count, int lanes, void* ws, size_t ws_bytes,
                                void* stream) {
  BatchPlan bp;
  TSVD_TRY(plan_batch(descs, count, lanes, &bp));
  if (count == 0) return TSVD_OK;
  if (!ws || ((uintptr_t)ws & 255) != 0) return TSVD_ERR_INVALID_ARG;
  if (ws_bytes < bp.lane_off[bp.lanes]) return TSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  if (bp.lanes == 1) {
    for (int i : bp.order) TSVD_TRY(rbk_one(descs[i], base, s));
    return TSVD_OK;
  }
  LanePool* lp = nullptr;
  TSVD_TRY(lane_pool(&lp));
  if (cudaEventRecord(lp->fork, s) != cudaSuccess) return TSVD_ERR_CUDA;
  for (int l = 0; l < bp.lanes; ++l)
    if (cudaStreamWaitEvent(lp->s[l], lp->fork, 0) != cudaSuccess) return TSVD_ERR_CUDA;
  int rc = TSVD_OK;
  for (int i : bp.order) {
    const int l = bp.lane_of[i];
    rc = rbk_one(descs[i], base + bp.lane_off[l], lp->s[l]);
    if (rc != TSVD_OK) break;
  }
  // join every lane back into the caller's stream, also after an error
  for (int l = 0; l < bp.lanes; ++l) {
    if (cudaEventRecord(lp->done[l], lp->s[l]) != cudaSuccess || cudaStreamWaitEvent(s, lp->done[l], 0) != cudaSuccess)
      rc = (rc == TSVD_OK) ? TSVD_ERR_CUDA : rc;
  }
  return rc;
}

extern "C" const char* tsvd_strerror(int code) {
  switch (code) {
    case TSVD_OK: return "ok";
    case TSVD_ERR_INVALID_ARG: return "invalid argument";
    case TSVD_ERR_WORKSPACE: return "workspace too small";
    case TSVD_ERR_CUDA: return "CUDA launch or API failure";
    case TSVD_ERR_UNSUPPORTED: return "size or mode beyond a kernel limit";
    case TSVD_ERR_NOT_CONVERGED: return "eigen solve produced a non-finite value";
    case TSVD_ERR_RANK_DEFICIENT: return "a Fourier slice is rank deficient (pseudoinverse by QR needs full rank)";
    default: return "unknown status";
  }
}

extern "C" int tsvd_version(void) { return 100; }
