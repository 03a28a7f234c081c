// linalg.cu -- small dense FP64 kernels, one problem per Fourier slice.
//
//  * CholeskyQR pieces for the block orthonormalisation of the Krylov basis
//    (the T-QR step of Alg. 2): Cholesky of a Gram matrix (optionally
//    shifted), a right triangular solve W <- W R^{-1}, and the replacement of
//    numerically dependent columns by fresh orthonormal directions.
//  * The Hermitian eigen-solve behind the small SVD of Alg. 2
//    ([U_c, S_c, V_c] = T-SVD(C) with C = Q^H X per slice): with
//    G = C C^H = U_c S_c^2 U_c^H, Householder reduction of G to tridiagonal
//    form, bisection (Sturm counts) for the R largest eigenvalues, inverse
//    iteration for their vectors and the back-transformation.
#include <float.h>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

__device__ __forceinline__ int pidx(int i, int j, int n) { return i * n - (i * (i - 1)) / 2 + (j - i); }

// ---------------------------------------------------------------------------
// Cholesky (upper, right-looking) of one nb x nb Gram matrix per CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_chol_upper(const double2* __restrict__ G, long ldg, long sG,
                                                    double2* __restrict__ Rm, long ldr, long sR, int nb, double shift,
                                                    uint32_t* __restrict__ dead_out) {
  extern __shared__ __align__(16) double2 S[];  // packed upper triangle
  __shared__ double dg[128];
  __shared__ double red[16];
  __shared__ uint32_t dmask[4];
  __shared__ double rjj;
  __shared__ int isdead;
  const int b = blockIdx.x, tid = threadIdx.x;
  G += (long)b * sG;
  Rm += (long)b * sR;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    if (j >= i) S[pidx(i, j, nb)] = G[(long)i * ldg + j];
  }
  if (tid < nb) dg[tid] = G[(long)tid * ldg + tid].x;
  if (tid < 4) dmask[tid] = 0;
  __syncthreads();
  const double trace = block_sum(tid < nb ? dg[tid] : 0.0, red);
  const double sft = (shift > 0.0) ? shift * trace : 0.0;
  if (tid < nb) S[pidx(tid, tid, nb)].x += sft;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      const double d = S[pidx(j, j, nb)].x;
      const bool dead = (shift > 0.0) ? !(d > 0.0) : !(d > 1e-12 * dg[j]);
      isdead = dead;
      rjj = dead ? 1.0 : sqrt(d);
      if (dead) dmask[j >> 5] |= 1u << (j & 31);
    }
    __syncthreads();
    const double r = rjj;
    const bool dead = isdead;
    for (int k = j + 1 + tid; k < nb; k += blockDim.x) {
      const int p = pidx(j, k, nb);
      S[p] = dead ? make_double2(0, 0) : cscale(S[p], 1.0 / r);
    }
    if (tid == 0) S[pidx(j, j, nb)] = make_double2(r, 0);
    __syncthreads();
    const int nt = nb - j - 1;
    for (int e = tid; e < nt * nt; e += blockDim.x) {
      const int i = j + 1 + e / nt, k = j + 1 + e % nt;
      if (k < i) continue;
      const double2 a = S[pidx(j, i, nb)], c = S[pidx(j, k, nb)];
      double2 t = S[pidx(i, k, nb)];
      // t -= conj(a) * c
      t.x -= a.x * c.x + a.y * c.y;
      t.y -= a.x * c.y - a.y * c.x;
      S[pidx(i, k, nb)] = t;
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e - i * nb;
    Rm[(long)i * ldr + k] = (k >= i) ? S[pidx(i, k, nb)] : make_double2(0, 0);
  }
  if (tid < 4) dead_out[b * 4 + tid] = dmask[tid];
}

int chol_upper(const double2* G, long ldg, long sG, double2* Rm, long ldr, long sR, int nb, int batch, double shift,
               uint32_t* dead, cudaStream_t s) {
  if (nb <= 0 || batch <= 0) return TSVD_OK;
  if (nb > 128) return TSVD_ERR_UNSUPPORTED;
  const size_t smem = (size_t)nb * (nb + 1) / 2 * sizeof(double2);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_chol_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_chol_upper<<<batch, 256, smem, s>>>(G, ldg, sG, Rm, ldr, sR, nb, shift, dead);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// ---------------------------------------------------------------------------
// W <- W R^{-1}: each thread solves x R = w for one row by forward
// substitution; R (packed) and the CTA's rows live in shared memory.
// ---------------------------------------------------------------------------
constexpr int TRSM_ROWS = 32;

__global__ void __launch_bounds__(TRSM_ROWS) k_trsm_right_upper(double2* __restrict__ W, long ldw, long sW,
                                                               const double2* __restrict__ Rm, long ldr, long sR,
                                                               int n1, int nb, const uint32_t* __restrict__ dead) {
  extern __shared__ __align__(16) double2 sm[];
  double2* Rp = sm;                                 // packed upper, nb(nb+1)/2
  double2* Ws = sm + nb * (nb + 1) / 2;             // [TRSM_ROWS][nb + 1]
  const int b = blockIdx.y, tid = threadIdx.x;
  const int r0 = blockIdx.x * TRSM_ROWS;
  W += (long)b * sW;
  Rm += (long)b * sR;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    if (j >= i) Rp[pidx(i, j, nb)] = Rm[(long)i * ldr + j];
  }
  const int ld = nb + 1;
  for (int e = tid; e < TRSM_ROWS * nb; e += blockDim.x) {
    const int r = e / nb, j = e - r * nb;
    Ws[r * ld + j] = (r0 + r < n1) ? W[(long)(r0 + r) * ldw + j] : make_double2(0, 0);
  }
  __syncthreads();
  uint32_t dm[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) dm[w] = dead[b * 4 + w];
  double2* x = Ws + tid * ld;
  for (int j = 0; j < nb; ++j) {
    double2 acc = x[j];
    for (int i = 0; i < j; ++i) {
      const double2 rij = Rp[pidx(i, j, nb)];
      const double2 xi = x[i];
      acc.x -= xi.x * rij.x - xi.y * rij.y;
      acc.y -= xi.x * rij.y + xi.y * rij.x;
    }
    const double2 rjj = Rp[pidx(j, j, nb)];
    const bool isdead = (dm[j >> 5] >> (j & 31)) & 1u;
    x[j] = isdead ? make_double2(0, 0) : cscale(acc, 1.0 / rjj.x);
  }
  __syncthreads();
  for (int e = tid; e < TRSM_ROWS * nb; e += blockDim.x) {
    const int r = e / nb, j = e - r * nb;
    if (r0 + r < n1) W[(long)(r0 + r) * ldw + j] = Ws[r * ld + j];
  }
}

int trsm_right_upper(double2* W, long ldw, long sW, const double2* Rm, long ldr, long sR, int n1, int nb, int batch,
                     const uint32_t* dead, cudaStream_t s) {
  if (nb <= 0 || n1 <= 0 || batch <= 0) return TSVD_OK;
  if (nb > 128) return TSVD_ERR_UNSUPPORTED;
  const size_t smem = ((size_t)nb * (nb + 1) / 2 + (size_t)TRSM_ROWS * (nb + 1)) * sizeof(double2);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_trsm_right_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(cdiv(n1, TRSM_ROWS), batch);
  k_trsm_right_upper<<<grid, TRSM_ROWS, smem, s>>>(W, ldw, sW, Rm, ldr, sR, n1, nb, dead);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// ---------------------------------------------------------------------------
// Dependent Krylov columns (exact low rank, zero data): replace column c+j by
// a Philox Gaussian direction (stream 3) projected twice against every other
// live column of the basis, then normalised.  Any orthonormal completion of
// span(K) leaves the Rayleigh-Ritz result of Alg. 2 optimal (eq. mn39).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_repair_dead(double2* __restrict__ Q, long ldq, long sQ, int n1, int c,
                                                     int nb, const uint32_t* __restrict__ dead, uint64_t seed,
                                                     int block_id, int* __restrict__ dead_count) {
  __shared__ double red[32];
  const int b = blockIdx.x, tid = threadIdx.x;
  uint32_t dm[4];
  int ndead = 0;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    dm[w] = dead[b * 4 + w];
    ndead += __popc(dm[w]);
  }
  if (ndead == 0) return;
  Q += (long)b * sQ;
  if (tid == 0) atomicAdd(dead_count, ndead);
  uint32_t pending[4] = {dm[0], dm[1], dm[2], dm[3]};
  for (int j = 0; j < nb; ++j) {
    if (!((dm[j >> 5] >> (j & 31)) & 1u)) continue;
    const int col = c + j;
    for (int attempt = 0; attempt < 4; ++attempt) {
      for (int i = tid; i < n1; i += blockDim.x) {
        const uint4 x = philox10(make_uint4((uint32_t)i, (uint32_t)col | ((uint32_t)attempt << 24),
                                            (uint32_t)block_id, 3u + ((uint32_t)b << 8)),
                                 (uint32_t)seed, (uint32_t)(seed >> 32));
        const double u1 = ((double)x.x + 1.0) * (1.0 / 4294967296.0);
        const double u2 = ((double)x.y + 1.0) * (1.0 / 4294967296.0);
        const double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        Q[(long)i * ldq + col] = make_double2(r * cs, r * sn);
      }
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int l = 0; l < c + nb; ++l) {
          if (l == col) continue;
          if (l >= c && ((pending[(l - c) >> 5] >> ((l - c) & 31)) & 1u)) continue;
          double2 part = make_double2(0, 0);
          for (int i = tid; i < n1; i += blockDim.x) cfmac(part, Q[(long)i * ldq + l], Q[(long)i * ldq + col]);
          const double2 dot = block_sum2(part, red);
          for (int i = tid; i < n1; i += blockDim.x) {
            double2 q = Q[(long)i * ldq + col];
            const double2 ql = Q[(long)i * ldq + l];
            q.x -= dot.x * ql.x - dot.y * ql.y;
            q.y -= dot.x * ql.y + dot.y * ql.x;
            Q[(long)i * ldq + col] = q;
          }
          __syncthreads();
        }
      }
      double part = 0;
      for (int i = tid; i < n1; i += blockDim.x) part += cabs2(Q[(long)i * ldq + col]);
      const double nrm = sqrt(block_sum(part, red));
      const bool ok = nrm > 1e-3;
      for (int i = tid; i < n1; i += blockDim.x)
        Q[(long)i * ldq + col] = ok ? cscale(Q[(long)i * ldq + col], 1.0 / nrm) : make_double2(0, 0);
      __syncthreads();
      if (ok) break;
    }
    pending[j >> 5] &= ~(1u << (j & 31));
  }
}

int repair_dead(double2* Q, long ldq, long sQ, int n1, int c, int nb, const uint32_t* dead, int batch, uint64_t seed,
                int block_id, int* dead_count, cudaStream_t s) {
  if (nb <= 0 || batch <= 0) return TSVD_OK;
  k_repair_dead<<<batch, 256, 0, s>>>(Q, ldq, sQ, n1, c, nb, dead, seed, block_id, dead_count);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// ---------------------------------------------------------------------------
// Hermitian eigen-solve, top R pairs.
// ---------------------------------------------------------------------------
struct EigScratch {
  double* d;        // [batch][m] diagonal of T
  double* f;        // [batch][m] off-diagonal |alpha_j|
  double2* alpha;   // [batch][m] complex off-diagonals
  double2* delta;   // [batch][m] phases making T real
  double2* Hv;      // [batch][m][m] Householder vectors (row j, columns j+1..m-1)
  double* Z;        // [batch][m][R] real eigenvectors of T
  double* lu;       // [batch][6][m][R] inverse-iteration work
  double* tnorm;    // [batch]
};

static EigScratch carve_eig(void* base, int m, int R, int batch, size_t* bytes) {
  Carver cv(base);
  EigScratch e;
  e.d = cv.take<double>((size_t)batch * m);
  e.f = cv.take<double>((size_t)batch * m);
  e.alpha = cv.take<double2>((size_t)batch * m);
  e.delta = cv.take<double2>((size_t)batch * m);
  e.Hv = cv.take<double2>((size_t)batch * m * m);
  e.Z = cv.take<double>((size_t)batch * m * R);
  e.lu = cv.take<double>((size_t)batch * 6 * m * R);
  e.tnorm = cv.take<double>((size_t)batch);
  if (bytes) *bytes = cv.bytes();
  return e;
}

size_t eig_scratch_bytes(int m, int R, int batch) {
  size_t b = 0;
  carve_eig(nullptr, m, R, batch, &b);
  return b;
}

// Householder reduction G -> T' = H_{m-2}..H_0 G H_0..H_{m-2} (Hermitian
// tridiagonal), one CTA per slice.  Step j: x = G(j+1:, j) (read as the
// conjugate of row j), alpha = -e^{i arg x_0} ||x||, v = (x - alpha e_1)
// normalised, p = 2 A v, w = p - (v^H p) v, A <- A - v w^H - w v^H on the
// trailing block (both triangles kept, so rows stay contiguous).
__global__ void __launch_bounds__(512) k_hetrd(double2* __restrict__ G, long ldg, long sG, int m, EigScratch e) {
  extern __shared__ __align__(16) double2 sh[];
  double2* v = sh;      // [m]
  double2* p = sh + m;  // [m]
  __shared__ double red[64];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  G += (long)b * sG;
  double2* Hv = e.Hv + (long)b * m * m;
  for (int j = 0; j < m - 1; ++j) {
    const int n = m - j - 1;
    const double2* rowj = G + (long)j * ldg + j + 1;
    double part = 0;
    for (int i = tid; i < n; i += blockDim.x) {
      const double2 x = cconj(rowj[i]);
      v[i] = x;
      part += cabs2(x);
    }
    const double nrm2 = block_sum(part, red);  // synchronises: v visible
    const double2 x0 = v[0];
    const double djj = G[(long)j * ldg + j].x;
    __syncthreads();
    if (tid == 0) e.d[(long)b * m + j] = djj;
    if (nrm2 == 0.0) {
      for (int i = tid; i < n; i += blockDim.x) Hv[(long)j * m + j + 1 + i] = make_double2(0, 0);
      if (tid == 0) e.alpha[(long)b * m + j] = make_double2(0, 0);
      __syncthreads();
      continue;
    }
    const double nrm = sqrt(nrm2), ax0 = sqrt(cabs2(x0));
    const double2 ph = (ax0 > 0) ? cscale(x0, 1.0 / ax0) : make_double2(1, 0);
    const double2 alpha = cscale(ph, -nrm);
    const double vinv = 1.0 / sqrt(2.0 * nrm * (nrm + ax0));
    for (int i = tid; i < n; i += blockDim.x) {
      double2 vi = v[i];
      if (i == 0) vi = csub(vi, alpha);
      vi = cscale(vi, vinv);
      v[i] = vi;
      Hv[(long)j * m + j + 1 + i] = vi;
    }
    if (tid == 0) e.alpha[(long)b * m + j] = alpha;
    __syncthreads();
    // p = 2 A22 v
    for (int r = warp; r < n; r += nwarp) {
      const double2* row = G + (long)(j + 1 + r) * ldg + j + 1;
      double2 acc = make_double2(0, 0);
      for (int k = lane; k < n; k += 32) cfma(acc, row[k], v[k]);
      acc = warp_sum(acc);
      if (lane == 0) p[r] = cscale(acc, 2.0);
    }
    __syncthreads();
    double2 kp = make_double2(0, 0);
    for (int i = tid; i < n; i += blockDim.x) cfmac(kp, v[i], p[i]);
    const double K = block_sum2(kp, red).x;
    for (int i = tid; i < n; i += blockDim.x) p[i] = csub(p[i], cscale(v[i], K));  // p <- w
    __syncthreads();
    for (long idx = tid; idx < (long)n * n; idx += blockDim.x) {
      const int r = (int)(idx / n), k = (int)(idx - (long)r * n);
      double2* g = G + (long)(j + 1 + r) * ldg + j + 1 + k;
      const double2 vr = v[r], wr = p[r], vk = v[k], wk = p[k];
      double2 t = *g;
      // t -= v_r conj(w_k) + w_r conj(v_k)
      t.x -= vr.x * wk.x + vr.y * wk.y + wr.x * vk.x + wr.y * vk.y;
      t.y -= vr.y * wk.x - vr.x * wk.y + wr.y * vk.x - wr.x * vk.y;
      *g = t;
    }
    __syncthreads();
  }
  if (tid == 0) {
    e.d[(long)b * m + m - 1] = G[(long)(m - 1) * ldg + m - 1].x;
    // phases: T = D^H T' D real with T(j+1, j) = |alpha_j|
    double2 dl = make_double2(1, 0);
    e.delta[(long)b * m] = dl;
    double tn = 0;
    for (int j = 0; j < m - 1; ++j) {
      const double2 a = e.alpha[(long)b * m + j];
      const double aa = sqrt(cabs2(a));
      e.f[(long)b * m + j] = aa;
      if (aa > 0) dl = cmul(dl, cscale(a, 1.0 / aa));
      e.delta[(long)b * m + j + 1] = dl;
    }
    for (int j = 0; j < m; ++j) {
      const double fl = (j > 0) ? e.f[(long)b * m + j - 1] : 0.0, fr = (j < m - 1) ? e.f[(long)b * m + j] : 0.0;
      tn = fmax(tn, fabs(e.d[(long)b * m + j]) + fl + fr);
    }
    e.tnorm[b] = tn;
  }
}

// number of eigenvalues of the real symmetric tridiagonal (d, f) below x
__device__ int sturm_count(const double* d, const double* f, int m, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = d[i] - x - f[i - 1] * f[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// One thread per (slice, r): the (r+1)-th largest eigenvalue of T by bisection,
// then its vector by inverse iteration with a partially pivoted LU of T - lam I.
__global__ void k_tridiag_pairs(int m, int R, int batch, EigScratch e, double* __restrict__ lam_out) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= batch * R) return;
  const int b = gid / R, r = gid - b * R;
  const double* d = e.d + (long)b * m;
  const double* f = e.f + (long)b * m;
  double lo = d[0], hi = d[0], fmax2 = 0;
  for (int i = 0; i < m; ++i) {
    const double fl = (i > 0) ? f[i - 1] : 0.0, fr = (i < m - 1) ? f[i] : 0.0;
    lo = fmin(lo, d[i] - fl - fr);
    hi = fmax(hi, d[i] + fl + fr);
    if (i < m - 1) fmax2 = fmax(fmax2, f[i] * f[i]);
  }
  const double tn = fmax(fabs(lo), fabs(hi));
  const double pivmin = DBL_MIN * fmax(1.0, fmax2);
  lo -= 2.0 * DBL_EPSILON * tn + pivmin;
  hi += 2.0 * DBL_EPSILON * tn + pivmin;
  const int idx = m - 1 - r;  // ascending index of the wanted eigenvalue
  for (int it = 0; it < 256; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 2.0 * DBL_EPSILON * (fabs(lo) + fabs(hi)) + pivmin || mid == lo || mid == hi) break;
    if (sturm_count(d, f, m, mid, pivmin) > idx) hi = mid;
    else lo = mid;
  }
  const double lam = 0.5 * (lo + hi);
  lam_out[(long)b * R + r] = lam;

  // work arrays, element i of array a at lu[((b*6 + a)*m + i)*R + r] (coalesced over r)
  double* base = e.lu + (long)b * 6 * m * R + r;
#define LU(a, i) base[((long)(a) * m + (i)) * R]
  // a: 0 dl (multipliers), 1 dd (U diagonal), 2 du (U first super), 3 du2 (U second super), 4 piv, 5 x
  const double tiny = DBL_EPSILON * fmax(tn, 1e-200);
  for (int i = 0; i < m; ++i) {
    LU(1, i) = d[i] - lam;
    LU(0, i) = (i < m - 1) ? f[i] : 0.0;
    LU(2, i) = (i < m - 1) ? f[i] : 0.0;
    LU(3, i) = 0.0;
  }
  for (int i = 0; i < m - 1; ++i) {
    const double a = LU(1, i), sub = LU(0, i);
    if (fabs(a) >= fabs(sub)) {
      const double piv = (fabs(a) < tiny) ? copysign(tiny, a) : a;
      LU(1, i) = piv;
      const double l = sub / piv;
      LU(0, i) = l;
      LU(1, i + 1) -= l * LU(2, i);
      LU(4, i) = 0.0;
    } else {
      // swap rows i and i+1: new row i = (sub, dd[i+1], du[i+1])
      const double sb = (fabs(sub) < tiny) ? copysign(tiny, sub) : sub;
      const double l = a / sb;
      const double dd1 = LU(1, i + 1), du0 = LU(2, i), du1 = (i < m - 2) ? LU(2, i + 1) : 0.0;
      LU(1, i) = sb;
      LU(2, i) = dd1;
      LU(3, i) = du1;
      LU(1, i + 1) = du0 - l * dd1;
      if (i < m - 2) LU(2, i + 1) = -l * du1;
      LU(0, i) = l;
      LU(4, i) = 1.0;
    }
  }
  if (fabs(LU(1, m - 1)) < tiny) LU(1, m - 1) = copysign(tiny, LU(1, m - 1));
  // starting vector: Philox uniforms in (-1, 1)
  for (int i = 0; i < m; ++i) {
    const uint4 x = philox10(make_uint4((uint32_t)i, (uint32_t)r, (uint32_t)b, 0x1e16u), 0x2504u, 0x4989u);
    LU(5, i) = ((double)x.x + 0.5) * (2.0 / 4294967296.0) - 1.0;
  }
  for (int iter = 0; iter < 3; ++iter) {
    // forward: apply the row interchanges and multipliers
    for (int i = 0; i < m - 1; ++i) {
      if (LU(4, i) != 0.0) {
        const double t = LU(5, i);
        LU(5, i) = LU(5, i + 1);
        LU(5, i + 1) = t;
      }
      LU(5, i + 1) -= LU(0, i) * LU(5, i);
    }
    // back substitution with U
    for (int i = m - 1; i >= 0; --i) {
      double s = LU(5, i);
      if (i + 1 < m) s -= LU(2, i) * LU(5, i + 1);
      if (i + 2 < m) s -= LU(3, i) * LU(5, i + 2);
      LU(5, i) = s / LU(1, i);
    }
    double mx = 0;
    for (int i = 0; i < m; ++i) mx = fmax(mx, fabs(LU(5, i)));
    if (!(mx > 0) || !isfinite(mx)) mx = 1.0;
    double nrm2 = 0;
    for (int i = 0; i < m; ++i) {
      const double t = LU(5, i) / mx;
      LU(5, i) = t;
      nrm2 += t * t;
    }
    const double inv = 1.0 / sqrt(nrm2);
    for (int i = 0; i < m; ++i) LU(5, i) *= inv;
  }
  double* Z = e.Z + (long)b * m * R;
  for (int i = 0; i < m; ++i) Z[(long)i * R + r] = LU(5, i);
#undef LU
}

// Within clusters of close eigenvalues (gap < 1e-3 ||T||) the independently
// iterated vectors are made orthonormal by two modified Gram-Schmidt passes.
__global__ void __launch_bounds__(256) k_cluster_orth(int m, int R, EigScratch e, const double* __restrict__ lam) {
  __shared__ double red[32];
  const int b = blockIdx.x, tid = threadIdx.x;
  double* Z = e.Z + (long)b * m * R;
  const double* l = lam + (long)b * R;
  const double tol = 1e-3 * e.tnorm[b];
  int c0 = 0;
  for (int r = 1; r < R; ++r) {
    if (l[r - 1] - l[r] > tol) {
      c0 = r;
      continue;
    }
    for (int pass = 0; pass < 2; ++pass) {
      for (int s = c0; s < r; ++s) {
        double part = 0;
        for (int i = tid; i < m; i += blockDim.x) part += Z[(long)i * R + s] * Z[(long)i * R + r];
        const double dot = block_sum(part, red);
        for (int i = tid; i < m; i += blockDim.x) Z[(long)i * R + r] -= dot * Z[(long)i * R + s];
        __syncthreads();
      }
      double part = 0;
      for (int i = tid; i < m; i += blockDim.x) part += Z[(long)i * R + r] * Z[(long)i * R + r];
      const double nrm = sqrt(block_sum(part, red));
      for (int i = tid; i < m; i += blockDim.x) Z[(long)i * R + r] /= nrm;
      __syncthreads();
    }
  }
}

// u_r = H_0 H_1 .. H_{m-2} D z_r, one warp per eigenvector.
constexpr int BT_WARPS = 8;
__global__ void __launch_bounds__(BT_WARPS * 32) k_backtransform(int m, int R, EigScratch e, double2* __restrict__ U,
                                                                 long ldu, long sU) {
  extern __shared__ __align__(16) double2 us[];
  const int b = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * BT_WARPS + warp;
  if (r >= R) return;
  double2* u = us + (long)warp * m;
  const double* Z = e.Z + (long)b * m * R;
  const double2* dl = e.delta + (long)b * m;
  const double2* Hv = e.Hv + (long)b * m * m;
  for (int i = lane; i < m; i += 32) u[i] = cscale(dl[i], Z[(long)i * R + r]);
  __syncwarp();
  for (int j = m - 2; j >= 0; --j) {
    const int n = m - j - 1;
    const double2* v = Hv + (long)j * m + j + 1;
    double2 acc = make_double2(0, 0);
    for (int i = lane; i < n; i += 32) cfmac(acc, v[i], u[j + 1 + i]);
    acc = warp_sum(acc);
    const double2 s2 = cscale(acc, 2.0);
    for (int i = lane; i < n; i += 32) u[j + 1 + i] = csub(u[j + 1 + i], cmul(v[i], s2));
    __syncwarp();
  }
  double2* Ub = U + (long)b * sU;
  for (int i = lane; i < m; i += 32) Ub[(long)i * ldu + r] = u[i];
}

int herm_eig_topR(double2* G, long ldg, long sG, int m, int R, int batch, double* lam, double2* U, long ldu, long sU,
                  void* scratch, int* status, cudaStream_t s) {
  (void)status;
  if (m <= 0 || R <= 0 || batch <= 0) return TSVD_OK;
  if (R > m || m > 1024) return TSVD_ERR_UNSUPPORTED;
  EigScratch e = carve_eig(scratch, m, R, batch, nullptr);
  const size_t smem_trd = 2 * (size_t)m * sizeof(double2);
  if (smem_trd > 48 * 1024) cudaFuncSetAttribute(k_hetrd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_trd);
  {
    TSVD_STAGE("eig_hetrd", s);
    k_hetrd<<<batch, 512, smem_trd, s>>>(G, ldg, sG, m, e);
    TSVD_LAUNCHED();
  }
  {
    TSVD_STAGE("eig_tridiag", s);
    k_tridiag_pairs<<<cdiv((long)batch * R, 64), 64, 0, s>>>(m, R, batch, e, lam);
    TSVD_LAUNCHED();
    k_cluster_orth<<<batch, 256, 0, s>>>(m, R, e, lam);
    TSVD_LAUNCHED();
  }
  const size_t smem_bt = (size_t)BT_WARPS * m * sizeof(double2);
  if (smem_bt > 48 * 1024)
    cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bt);
  TSVD_STAGE("eig_backtransform", s);
  k_backtransform<<<dim3(cdiv(R, BT_WARPS), batch), BT_WARPS * 32, smem_bt, s>>>(m, R, e, U, ldu, sU);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_sigma(const double* __restrict__ lam, int n, double* __restrict__ sig, cx_t<T>* __restrict__ Sh,
                        int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l = lam[i];
  if (!isfinite(l)) atomicExch(status, TSVD_ERR_NOT_CONVERGED);
  const double sg = sqrt(fmax(l, 0.0));
  if (sig) sig[i] = sg;
  Sh[i] = mkc((T)sg, T(0));
}

template <typename T>
int sigma_from_lambda(const double* lam, int R, int batch, double* sig, cx_t<T>* Sh, cudaStream_t s, int* status) {
  const int n = R * batch;
  if (n <= 0) return TSVD_OK;
  k_sigma<T><<<cdiv(n, 256), 256, 0, s>>>(lam, n, sig, Sh, status);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int sigma_from_lambda<double>(const double*, int, int, double*, double2*, cudaStream_t, int*);
template int sigma_from_lambda<float>(const double*, int, int, double*, float2*, cudaStream_t, int*);

template <typename T>
__global__ void k_scale_cols(cx_t<T>* __restrict__ V, long ldv, long sV, int rows, int R,
                             const double* __restrict__ lam, int batch) {
  const long total = (long)batch * rows * R;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int r = idx % R;
    const long t = idx / R;
    const int i = t % rows;
    const int b = t / rows;
    const double sg = sqrt(fmax(lam[(long)b * R + r], 0.0));
    const T inv = (sg > 0.0) ? (T)(1.0 / sg) : T(0);
    cx_t<T>* p = V + (long)b * sV + (long)i * ldv + r;
    *p = cscale(*p, inv);
  }
}

template <typename T>
int scale_columns_inv(cx_t<T>* V, long ldv, long sV, int rows, int R, const double* lam, int batch, cudaStream_t s) {
  const long total = (long)batch * rows * R;
  if (total <= 0) return TSVD_OK;
  k_scale_cols<T><<<std::min<long>(cdiv(total, 256), 8192), 256, 0, s>>>(V, ldv, sV, rows, R, lam, batch);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int scale_columns_inv<double>(double2*, long, long, int, int, const double*, int, cudaStream_t);
template int scale_columns_inv<float>(float2*, long, long, int, int, const double*, int, cudaStream_t);

}  // namespace tsvd
