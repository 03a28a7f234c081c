// eig.cu -- the Hermitian eigen-solve behind the small SVD of Alg. 2
// ([U_c, S_c, V_c] = T-SVD(C) with C = Q^H X per Fourier slice): with
// G = C C^H = U_c S_c^2 U_c^H, the R largest eigenpairs of the m x m G give
// sigma_i = sqrt(lambda_i) and U_c(:, 1:R).
//
//   1. Householder reduction to tridiagonal form, T' = H_{m-2}..H_0 G H_0..H_{m-2};
//      a cluster of CTAs shares each slice's rows (FP64 is the bound, so the
//      work of one slice is spread over several SMs).
//   2. T = D^H T' D real symmetric (D diagonal unitary); bisection on Sturm
//      counts (a division-free three-term recurrence) for the R largest
//      eigenvalues, inverse iteration with a partially pivoted LU for the
//      vectors, two classical Gram-Schmidt passes inside clusters of close
//      eigenvalues.
//   3. u_r = H_0 .. H_{m-2} D z_r.
#include <cooperative_groups.h>
#include <float.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace tsvd {

struct EigScratch {
  double* d;       // [batch][m] diagonal of T
  double* f;       // [batch][m] off-diagonal |alpha_j|
  double2* alpha;  // [batch][m] complex off-diagonals of T'
  double2* delta;  // [batch][m] phases making T real
  double2* Hv;     // [batch][m][m] Householder vectors (row j, columns j+1..m-1)
  double2* pbuf;   // [batch][m] matrix-vector product shared inside a cluster
  double* Z;       // [batch][m][R] real eigenvectors of T
  double* lu;      // [batch][6][m][R] inverse-iteration work
  double* tnorm;   // [batch]
};

static EigScratch carve_eig(void* base, int m, int R, int batch, size_t* bytes) {
  Carver cv(base);
  EigScratch e;
  e.d = cv.take<double>((size_t)batch * m);
  e.f = cv.take<double>((size_t)batch * m);
  e.alpha = cv.take<double2>((size_t)batch * m);
  e.delta = cv.take<double2>((size_t)batch * m);
  e.Hv = cv.take<double2>((size_t)batch * m * m);
  e.pbuf = cv.take<double2>((size_t)batch * m);
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

__device__ __forceinline__ double2 ldcg2(const double2* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Householder tridiagonalisation, one cluster of CL CTAs per slice.  Rows of
// the trailing block are owned round-robin (global row g by CTA g mod CL).
// Step j: every CTA reads row j (x = conj of it) and forms the same
// v = (x - alpha e_1)/||.||, alpha = -e^{i arg x_0} ||x||; each CTA computes
// p = 2 A v on its rows; after a cluster barrier every CTA reads all of p,
// forms w = p - (v^H p) v and updates its rows A -= v w^H + w v^H (both
// triangles, so rows stay contiguous).  Data another CTA wrote is read with
// L2-coherent loads after the barrier (release / acquire at cluster scope).
// ---------------------------------------------------------------------------
template <int CL>
__global__ void __launch_bounds__(512) k_hetrd(double2* __restrict__ G, long ldg, long sG, int m, EigScratch e) {
  extern __shared__ __align__(16) double2 sh[];
  double2* v = sh;      // [m]
  double2* p = sh + m;  // [m]
  __shared__ double red[64];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (CL > 1) ? (int)cluster.block_rank() : 0;
  const int b = blockIdx.x / CL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  G += (long)b * sG;
  double2* Hv = e.Hv + (long)b * m * m;
  double2* pb = e.pbuf + (long)b * m;
  for (int j = 0; j < m - 1; ++j) {
    const int n = m - j - 1;
    const double2* rowj = G + (long)j * ldg + j + 1;
    double part = 0;
    for (int i = tid; i < n; i += blockDim.x) {
      const double2 x = cconj(ldcg2(rowj + i));
      v[i] = x;
      part += cabs2(x);
    }
    const double nrm2 = block_sum(part, red);  // synchronises: v visible
    const double2 x0 = v[0];
    const double djj = ldcg2(G + (long)j * ldg + j).x;
    __syncthreads();
    if (rank == 0 && tid == 0) e.d[(long)b * m + j] = djj;
    const bool skip = !(nrm2 > 0.0);  // identical in every CTA of the cluster
    if (!skip) {
      const double nrm = sqrt(nrm2), ax0 = sqrt(cabs2(x0));
      const double2 ph = (ax0 > 0) ? cscale(x0, 1.0 / ax0) : make_double2(1, 0);
      const double2 alpha = cscale(ph, -nrm);
      const double vinv = 1.0 / sqrt(2.0 * nrm * (nrm + ax0));
      for (int i = tid; i < n; i += blockDim.x) {
        double2 vi = v[i];
        if (i == 0) vi = csub(vi, alpha);
        vi = cscale(vi, vinv);
        v[i] = vi;
        if (rank == 0) Hv[(long)j * m + j + 1 + i] = vi;
      }
      if (rank == 0 && tid == 0) e.alpha[(long)b * m + j] = alpha;
      __syncthreads();
      // p = 2 A v on the rows this CTA owns: global row g = j+1+r with g % CL == rank
      const int r0 = ((rank - (j + 1)) % CL + CL) % CL;
      for (int r = r0 + warp * CL; r < n; r += nwarp * CL) {
        const double2* row = G + (long)(j + 1 + r) * ldg + j + 1;
        double2 acc = make_double2(0, 0);
        for (int k = lane; k < n; k += 32) cfma(acc, row[k], v[k]);
        acc = warp_sum(acc);
        if (lane == 0) __stcg(pb + r, cscale(acc, 2.0));
      }
    } else {
      for (int i = tid; i < n; i += blockDim.x)
        if (rank == 0) Hv[(long)j * m + j + 1 + i] = make_double2(0, 0);
      if (rank == 0 && tid == 0) e.alpha[(long)b * m + j] = make_double2(0, 0);
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();
    if (!skip) {
      double2 kp = make_double2(0, 0);
      for (int i = tid; i < n; i += blockDim.x) {
        const double2 pi = ldcg2(pb + i);
        p[i] = pi;
        cfmac(kp, v[i], pi);
      }
      const double K = block_sum2(kp, red).x;
      for (int i = tid; i < n; i += blockDim.x) p[i] = csub(p[i], cscale(v[i], K));  // p <- w
      __syncthreads();
      const int r0 = ((rank - (j + 1)) % CL + CL) % CL;
      const int nown = (n > r0) ? (n - r0 + CL - 1) / CL : 0;
      for (long idx = tid; idx < (long)nown * n; idx += blockDim.x) {
        const int r = r0 + (int)(idx / n) * CL, k = (int)(idx % n);
        double2* g = G + (long)(j + 1 + r) * ldg + j + 1 + k;
        const double2 vr = v[r], wr = p[r], vk = v[k], wk = p[k];
        double2 t = *g;
        // t -= v_r conj(w_k) + w_r conj(v_k)
        t.x -= vr.x * wk.x + vr.y * wk.y + wr.x * vk.x + wr.y * vk.y;
        t.y -= vr.y * wk.x - vr.x * wk.y + wr.y * vk.x - wr.x * vk.y;
        *g = t;
      }
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();
  }
  if (rank == 0 && tid == 0) {
    e.d[(long)b * m + m - 1] = ldcg2(G + (long)(m - 1) * ldg + m - 1).x;
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

// Number of eigenvalues below x of the symmetric tridiagonal (d, f) (scaled
// to norm ~1): sign changes of the Sturm sequence P_0 = 1, P_1 = d_0 - x,
// P_i = (d_{i-1} - x) P_{i-1} - f_{i-2}^2 P_{i-2}, i.e. negative ratios
// q_i = P_i / P_{i-1}; a zero ratio is replaced by -pivmin.  The pair
// (P_i, P_{i-1}) is rescaled by powers of two to stay in range.
__device__ int sturm_count(const double* d, const double* f2, int m, double x, double pivmin) {
  double pm = 1.0, p = d[0] - x;
  if (p == 0.0) p = -pivmin;
  int cnt = (p < 0.0);
  for (int i = 1; i < m; ++i) {
    double pn = (d[i] - x) * p - f2[i - 1] * pm;
    if (pn == 0.0) pn = -pivmin * p;
    cnt += ((pn < 0.0) != (p < 0.0));
    pm = p;
    p = pn;
    const double s = fabs(p) + fabs(pm);
    if (s > 0x1p+600) {
      p *= 0x1p-600;
      pm *= 0x1p-600;
    } else if (s < 0x1p-600) {
      p *= 0x1p+600;
      pm *= 0x1p+600;
    }
  }
  return cnt;
}

// One CTA per slice, one thread per wanted eigenpair r < R (the (r+1)-th
// largest): bisection, then inverse iteration (three solves).
__global__ void __launch_bounds__(128) k_tridiag_pairs(int m, int R, EigScratch e, double* __restrict__ lam_out) {
  extern __shared__ __align__(16) double tsm[];
  double* d = tsm;       // [m] scaled diagonal
  double* f = tsm + m;   // [m] scaled off-diagonal
  double* f2 = f + m;    // [m] squares
  __shared__ double s_scale;
  const int b = blockIdx.x, r = threadIdx.x;
  if (r == 0) {
    const double tn = e.tnorm[b];
    s_scale = (tn > 0.0 && isfinite(tn)) ? 1.0 / tn : 1.0;
  }
  __syncthreads();
  const double sc = s_scale;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    d[i] = e.d[(long)b * m + i] * sc;
    const double fi = (i < m - 1) ? e.f[(long)b * m + i] * sc : 0.0;
    f[i] = fi;
    f2[i] = fi * fi;
  }
  __syncthreads();
  if (r >= R) return;
  if (!(e.tnorm[b] > 0.0)) {  // T = 0 (zero data): every eigenvalue is 0, vectors e_r
    lam_out[(long)b * R + r] = 0.0;
    double* Z0 = e.Z + (long)b * m * R;
    for (int i = 0; i < m; ++i) Z0[(long)i * R + r] = (i == r) ? 1.0 : 0.0;
    return;
  }
  double lo = d[0], hi = d[0];
  for (int i = 0; i < m; ++i) {
    const double fl = (i > 0) ? f[i - 1] : 0.0, fr = f[i];
    lo = fmin(lo, d[i] - fl - fr);
    hi = fmax(hi, d[i] + fl + fr);
  }
  const double tn = fmax(fabs(lo), fabs(hi));
  const double pivmin = DBL_MIN * 0x1p+64;
  lo -= 4.0 * DBL_EPSILON * tn + pivmin;
  hi += 4.0 * DBL_EPSILON * tn + pivmin;
  const int idx = m - 1 - r;  // ascending index of the wanted eigenvalue
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 2.0 * DBL_EPSILON * (fabs(lo) + fabs(hi)) + pivmin || mid == lo || mid == hi) break;
    if (sturm_count(d, f2, m, mid, pivmin) > idx) hi = mid;
    else lo = mid;
  }
  const double lam = 0.5 * (lo + hi);
  lam_out[(long)b * R + r] = lam / sc;

  // element i of work array a at lu[((b*6 + a)*m + i)*R + r] (coalesced over r)
  double* base = e.lu + (long)b * 6 * m * R + r;
#define LU(a, i) base[((long)(a) * m + (i)) * R]
  // a: 0 multipliers, 1 reciprocal U diagonal, 2 U first super, 3 U second super, 4 row swap, 5 x
  const double tiny = DBL_EPSILON * fmax(tn, 1e-200);
  for (int i = 0; i < m; ++i) {
    LU(1, i) = d[i] - lam;
    LU(0, i) = f[i];
    LU(2, i) = f[i];
    LU(3, i) = 0.0;
  }
  for (int i = 0; i < m - 1; ++i) {
    const double a = LU(1, i), sub = LU(0, i);
    if (fabs(a) >= fabs(sub)) {
      const double piv = (fabs(a) < tiny) ? copysign(tiny, a) : a;
      const double l = sub / piv;
      LU(1, i) = 1.0 / piv;
      LU(0, i) = l;
      LU(1, i + 1) -= l * LU(2, i);
      LU(4, i) = 0.0;
    } else {
      // swap rows i and i+1: the new row i is (sub, d_{i+1}, du_{i+1})
      const double sb = (fabs(sub) < tiny) ? copysign(tiny, sub) : sub;
      const double l = a / sb;
      const double dd1 = LU(1, i + 1), du0 = LU(2, i), du1 = (i < m - 2) ? LU(2, i + 1) : 0.0;
      LU(1, i) = 1.0 / sb;
      LU(2, i) = dd1;
      LU(3, i) = du1;
      LU(1, i + 1) = du0 - l * dd1;
      if (i < m - 2) LU(2, i + 1) = -l * du1;
      LU(0, i) = l;
      LU(4, i) = 1.0;
    }
  }
  {
    const double a = LU(1, m - 1);
    LU(1, m - 1) = 1.0 / ((fabs(a) < tiny) ? copysign(tiny, a) : a);
  }
  for (int i = 0; i < m; ++i) {  // starting vector: Philox uniforms in (-1, 1)
    const uint4 x = philox10(make_uint4((uint32_t)i, (uint32_t)r, (uint32_t)b, 0x1e16u), 0x2504u, 0x4989u);
    LU(5, i) = ((double)x.x + 0.5) * (2.0 / 4294967296.0) - 1.0;
  }
  for (int iter = 0; iter < 3; ++iter) {
    for (int i = 0; i < m - 1; ++i) {  // row interchanges and multipliers
      if (LU(4, i) != 0.0) {
        const double t = LU(5, i);
        LU(5, i) = LU(5, i + 1);
        LU(5, i + 1) = t;
      }
      LU(5, i + 1) -= LU(0, i) * LU(5, i);
    }
    double mx = 0;
    for (int i = m - 1; i >= 0; --i) {  // back substitution with U
      double s = LU(5, i);
      if (i + 1 < m) s -= LU(2, i) * LU(5, i + 1);
      if (i + 2 < m) s -= LU(3, i) * LU(5, i + 2);
      s *= LU(1, i);
      LU(5, i) = s;
      mx = fmax(mx, fabs(s));
    }
    if (!(mx > 0) || !isfinite(mx)) mx = 1.0;
    const double imx = 1.0 / mx;
    double nrm2 = 0;
    for (int i = 0; i < m; ++i) {
      const double t = LU(5, i) * imx;
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

// Inside clusters of close eigenvalues (gap < 1e-3 ||T||) the vectors are
// made orthonormal: two classical Gram-Schmidt passes against the earlier
// members of the cluster, then normalisation.
__global__ void __launch_bounds__(256) k_cluster_orth(int m, int R, EigScratch e, const double* __restrict__ lam) {
  __shared__ double red[32];
  __shared__ double dots[128];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
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
      for (int s = c0 + warp; s < r; s += nwarp) {
        double acc = 0;
        for (int i = lane; i < m; i += 32) acc += Z[(long)i * R + s] * Z[(long)i * R + r];
        acc = warp_sum(acc);
        if (lane == 0) dots[s - c0] = acc;
      }
      __syncthreads();
      for (int i = tid; i < m; i += blockDim.x) {
        double acc = Z[(long)i * R + r];
        for (int s = c0; s < r; ++s) acc -= dots[s - c0] * Z[(long)i * R + s];
        Z[(long)i * R + r] = acc;
      }
      __syncthreads();
    }
    double part = 0;
    for (int i = tid; i < m; i += blockDim.x) part += Z[(long)i * R + r] * Z[(long)i * R + r];
    const double nrm = sqrt(block_sum(part, red));
    for (int i = tid; i < m; i += blockDim.x) Z[(long)i * R + r] /= nrm;
    __syncthreads();
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

constexpr int HETRD_CLUSTER = 4;

int herm_eig_topR(double2* G, long ldg, long sG, int m, int R, int batch, double* lam, double2* U, long ldu, long sU,
                  void* scratch, int* status, cudaStream_t s) {
  (void)status;
  if (m <= 0 || R <= 0 || batch <= 0) return TSVD_OK;
  if (R > m || R > 128 || m > 1024) return TSVD_ERR_UNSUPPORTED;
  EigScratch e = carve_eig(scratch, m, R, batch, nullptr);
  {
    TSVD_STAGE("eig_hetrd", s);
    const size_t smem = 2 * (size_t)m * sizeof(double2);
    if (smem > 48 * 1024) {
      cudaFuncSetAttribute(k_hetrd<HETRD_CLUSTER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(batch * HETRD_CLUSTER);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = HETRD_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_hetrd<HETRD_CLUSTER>, G, ldg, sG, m, e) != cudaSuccess) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    TSVD_LAUNCHED();
  }
  {
    TSVD_STAGE("eig_tridiag", s);
    k_tridiag_pairs<<<batch, 128, 3 * (size_t)m * sizeof(double), s>>>(m, R, e, lam);
    TSVD_LAUNCHED();
    k_cluster_orth<<<batch, 256, 0, s>>>(m, R, e, lam);
    TSVD_LAUNCHED();
  }
  TSVD_STAGE("eig_backtransform", s);
  const size_t smem_bt = (size_t)BT_WARPS * m * sizeof(double2);
  if (smem_bt > 48 * 1024)
    cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bt);
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
