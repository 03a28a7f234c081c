// deflate.cu -- deflated Rayleigh-Ritz passes for the small SVD of Alg. 2 on
// the FP64 path (TSVD_FLAG_DEFLATE).
//
// The small SVD goes through the Gram G = C C^H, whose eigenvalues a
// backward-stable solver returns to an absolute accuracy of ~eps lambda_1:
// singular values below ~1e-8 sigma_1 are lost.  Spectra such as the paper's
// Ex. 1 (Sec. 5: sigma_m = m^-5, m^-6, 0.5^m) keep R = 45 values far below
// that.  Each pass therefore accepts the eigenpairs it resolves (lambda >=
// 1e-6 lambda_max of the pass, accurate to ~1e-10 relative), projects their
// directions out of C twice (C <- (I - U_a U_a^H) C, as classical
// Gram-Schmidt twice), and solves the Gram of the remainder, whose largest
// eigenvalue is the next unresolved one.  Every pass extends the resolved
// range by six decades of lambda; the singular values end with the absolute
// accuracy ~eps sigma_1 that the FP64 C itself carries.
#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

constexpr double DEFLATE_TAU = 1e-6;

// One block per slice.  The pass's eigenpairs (lam_p: R values descending,
// U_p: mp x R) extend the accepted set (lamF, UF, and Um = the accepted
// columns with zeros beyond): those with lambda >= tau * lambda_max, or all
// that are still missing on the last pass.  acc holds the accepted count.
__global__ void __launch_bounds__(256) k_deflate_merge(const double* __restrict__ lam_p,
                                                       const double2* __restrict__ U_p, int mp, int R,
                                                       double* __restrict__ lamF, double2* __restrict__ UF,
                                                       double2* __restrict__ Um, int* __restrict__ acc, int first,
                                                       int last) {
  __shared__ int s_a, s_t;
  const int b = blockIdx.x, tid = threadIdx.x;
  lam_p += (long)b * R;
  lamF += (long)b * R;
  U_p += (long)b * mp * R;
  UF += (long)b * mp * R;
  Um += (long)b * mp * R;
  if (tid == 0) {
    const int a = first ? 0 : acc[b];
    const int rem = R - a;
    const double lmax = lam_p[0];
    int t = 0;
    if (last || !(lmax > 0.0)) t = rem;
    else
      while (t < rem && lam_p[t] >= DEFLATE_TAU * lmax) ++t;
    s_a = a;
    s_t = t;
    acc[b] = a + t;
  }
  __syncthreads();
  const int a = s_a, t = s_t;
  for (int i = tid; i < t; i += blockDim.x) lamF[a + i] = lam_p[i];
  for (long e = tid; e < (long)mp * t; e += blockDim.x) {
    const int r = (int)(e / t), i = (int)(e % t);
    const double2 u = U_p[(long)r * R + i];
    UF[(long)r * R + a + i] = u;
    Um[(long)r * R + a + i] = u;
  }
}

int deflate_merge(const double* lam_p, const double2* U_p, int mp, int R, int batch, double* lamF, double2* UF,
                  double2* Um, int* acc, bool first, bool last, cudaStream_t s) {
  if (batch <= 0 || R <= 0) return TSVD_OK;
  k_deflate_merge<<<batch, 256, 0, s>>>(lam_p, U_p, mp, R, lamF, UF, Um, acc, first ? 1 : 0, last ? 1 : 0);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
